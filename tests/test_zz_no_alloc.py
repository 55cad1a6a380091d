"""The allocation-free sort entry point (pic_sort_cells_noalloc) must give the
same result as the context's sort (pic_sort) for callers that cannot give the
library device memory of their own.  Collected last on purpose: it runs after
every other test, and must also pass alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest

from tests import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as G
    G.build()


def _sorted_key(st):
    o = np.lexsort((st["id"], st["cell"]))
    return {k: v[o] for k, v in st.items()}


def test_noalloc_sort_matches_context_sort_twice():
    import paper_2212_08836_gb300 as P

    nr, nz, n = 64, 96, 200000
    rng = np.random.default_rng(7)
    e = inputs.particles(nr, nz, n, 70, 1e5, sorted_=False)
    e["cell"][rng.random(n) < 0.03] = -1
    i = inputs.particles(nr, nz, n, 71, 1e3, sorted_=False)
    cfg = P.small_reactor(nr=nr, nz=nz, np_init=n, capacity_factor=1.0, mcc_on=0)
    pic = P.Pic(cfg, device=DEV)
    pic.set_state([e, i])
    v = pic.view()
    src = {k: v["species"][0][k][:n].clone() for k in P.FIELDS}  # unsorted electrons
    pic.sort()  # the existing entry point (context workspace)
    ref = _sorted_key(pic.get_state(0))
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = {k: torch.full_like(src[k], -7) for k in P.FIELDS}
        n_out = C.c_longlong(-1)
        args = [nr, nz, n] + [src[k].data_ptr() for k in P.FIELDS] + \
               [out[k].data_ptr() for k in P.FIELDS] + [stream, C.addressof(n_out)]
        torch.cuda.synchronize()
        held, free = torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0]
        rc = P.lib().pic_sort_cells_noalloc(*args)
        assert rc == 0, P.lib().pic_strerror(rc)
        torch.cuda.synchronize()
        if call == 1:
            # the first call may load the module's static array; later calls
            # take no device memory at all
            assert torch.cuda.memory_allocated() == held
            assert torch.cuda.mem_get_info()[0] == free
        m = n_out.value
        assert m == len(ref["cell"])
        got = {k: out[k][:m].cpu().numpy() for k in P.FIELDS}
        got["id"] = got["id"].view(np.uint32)
        assert np.all(np.diff(got["cell"]) >= 0)
        got = _sorted_key(got)
        for k in P.FIELDS:
            np.testing.assert_array_equal(got[k], ref[k], err_msg="call %d %s" % (call, k))


def test_noalloc_sort_rejects_grids_beyond_its_limit():
    import paper_2212_08836_gb300 as P

    n_out = C.c_longlong(-1)
    rc = P.lib().pic_sort_cells_noalloc(1024, 1024, 0, *([None] * 16), None, C.addressof(n_out))
    assert rc == P.PIC_E_CONFIG
