"""The FP64 mover's integer-pipe binary64 multiply (csrc/swfp.cuh) is the IEEE
binary64 multiply: on the host (its source compiled as C++) and on the GPU
(through pic_check_dmul) it agrees bit for bit with the IEEE multiply, round to
nearest even, over the exponent range, exact and tie cases, subnormal and
overflowing results and the special values."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_host_build_matches_ieee_multiply(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path / "swfp_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "swfp_host_check.cpp")], check=True)
    r = subprocess.run([exe, "3000000"], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "mismatches 0" in r.stdout


def _operands(n, seed):
    """Random binary64 operand pairs (as in the host check): the exponent range,
    few-significand-bit cases, subnormal and overflowing products, specials."""
    rng = np.random.default_rng(seed)
    def rnd(emin, emax, k):
        m = rng.integers(0, 1 << 52, size=k, dtype=np.uint64)
        sel = rng.integers(0, 4, size=k)
        m = np.where(sel == 0, m & np.uint64(0x000FFF0000000000), m)
        m = np.where(sel == 1, m & np.uint64(0x000FFFFFFF000000), m)
        e = rng.integers(emin, emax + 1, size=k).astype(np.uint64)
        s = rng.integers(0, 2, size=k).astype(np.uint64) << np.uint64(63)
        return (s | (e << np.uint64(52)) | m).view(np.float64)
    q = n // 4
    x = np.concatenate([rnd(1, 2046, q), rnd(900, 1150, q), rnd(1, 80, q), rnd(1500, 2046, q)])
    y = np.concatenate([rnd(1, 2046, q), rnd(900, 1150, q), rnd(900, 1000, q), rnd(1000, 1100, q)])
    sp = np.array([0.0, -0.0, 1.0, -1.5, 5e-324, 2.2250738585072014e-308, 1e-310,
                   1.7976931348623157e308, np.inf, -np.inf, np.nan, 3e-200])
    xs, ys = np.meshgrid(sp, sp)
    return np.concatenate([x, xs.ravel()]), np.concatenate([y, ys.ravel()])


@pytest.mark.gpu
def test_gpu_multiply_is_bit_identical_to_ieee():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as G
    G.build()
    import paper_2212_08836_gb300 as M
    x, y = _operands(1 << 22, 5)
    with np.errstate(all="ignore"):
        ref = x * y
    got = M.check_dmul(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()).cpu().numpy()
    same = (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), (x[~same][:3], y[~same][:3], got[~same][:3], ref[~same][:3])
