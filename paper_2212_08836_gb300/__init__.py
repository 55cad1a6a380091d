"""GB300 (sm_103a) hot path of the implicit energy- and charge-conserving
EM PIC/MCC method of arXiv:2212.08836 — Python binding.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libpic.so`` (C ABI in ``include/pic.h``).  PyTorch provides the device
workspace and the stream.  There is no CPU fallback: importing the binding
without the compiled library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpic.so")

PIC_OK = 0
PIC_E_CONFIG = -1
PIC_E_CUDA = -2
PIC_E_NOCONV = -3
PIC_E_SUBSTEP = -4
PIC_E_CAPACITY = -5
PIC_E_NAN = -6
PIC_E_STATE = -7
PIC_E_WORKSPACE = -8
PIC_E_IO = -9
PIC_DIAG_ENERGY, PIC_DIAG_GAUSS, PIC_DIAG_CONTINUITY, PIC_DIAG_DENSITY_AVG = 0, 1, 2, 3
PIC_DIAG_ION_FLUX_AVG, PIC_DIAG_FIELDS, PIC_DIAG_COUNTS = 4, 5, 6
PIC_FEED_GAP = 0
PIC_FEED_WAVE = 1
PIC_FEED_AXIAL = 2
PIC_FP64 = 0
PIC_MIXED = 1

_P = C.c_void_p
_D = C.c_double
_I = C.c_int
_LL = C.c_longlong


class Config(C.Structure):
    _fields_ = [("nr", _I), ("nz", _I), ("R", _D), ("L", _D), ("dt", _D), ("freq", _D),
                ("volt", _D), ("gas_pressure", _D), ("gas_temp", _D), ("n0", _D),
                ("te_ev", _D), ("ti_ev", _D), ("np_init", _LL), ("capacity_factor", _D),
                ("picard_tol", _D), ("picard_max", _I), ("mcc_on", _I), ("bz", _D),
                ("eps", _D), ("mu", _D), ("seed", C.c_ulonglong), ("precision", _I),
                ("field_model", _I), ("cblock", _D), ("ions_fixed", _I), ("feed", _I),
                ("ring_cells", _I), ("eps_ring", _D), ("axis_cells", _I),
                ("sigma_ring", _D), ("port_cells", _I), ("port_len", _D), ("port_rin", _I),
                ("eps_port", _D), ("port_grade", _D)]


class StepStats(C.Structure):
    _fields_ = [("picard_iters", _I), ("converged", _I), ("last_res", _D), ("src_energy", _D),
                ("ke_lost", _D), ("de_coll", _D), ("substep_err", _LL), ("absorbed", _LL),
                ("substeps", _LL), ("fallbacks", _LL), ("mcc", _LL * 8), ("n", _LL * 2),
                ("pushes", _LL), ("launches", _LL), ("push_flops", _LL), ("guess", _I),
                ("spec_final", _I), ("first_res", _D), ("v_electrode", _D), ("q_cap", _D)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("mcc", "n")}
        d["mcc"] = list(self.mcc)
        d["n"] = list(self.n)
        return d


class CnnConfig(C.Structure):
    _fields_ = [("nr", _I), ("nz", _I), ("width", _I), ("depth", _I), ("batch", _I),
                ("seed", C.c_ulonglong)]


class HostState(C.Structure):
    _fields_ = [("n", _LL * 2), ("next_id", C.c_uint32 * 2), ("step", _LL),
                ("cell", _P * 2), ("a", _P * 2), ("b", _P * 2), ("vr", _P * 2), ("vt", _P * 2),
                ("vz", _P * 2), ("w", _P * 2), ("id", _P * 2), ("er", _P), ("ez", _P), ("h", _P)]


class View(C.Structure):
    _fields_ = [("cell", _P * 2), ("a", _P * 2), ("b", _P * 2), ("vr", _P * 2), ("vt", _P * 2),
                ("vz", _P * 2), ("w", _P * 2), ("id", _P * 2), ("n", _LL * 2), ("cap", _LL * 2),
                ("next_id", C.c_uint32 * 2), ("er", _P), ("ez", _P), ("h", _P), ("step", _LL),
                ("real_size", _I), ("wall", _P), ("qcond", _P), ("port_h", _P),
                ("port_er", _P), ("port_ez", _P), ("port_m", _I), ("port_cells", _I)]


class DiagOut(C.Structure):
    _fields_ = [("kinetic", _D * 2), ("field", _D), ("charge", _D * 2), ("n", _LL * 2)]


def _load_lib():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libpic.so is not built (run __graft_entry__.build() or "
                          "python paper_2212_08836_gb300/build.py); there is no CPU fallback")
    L = C.CDLL(LIB_PATH)
    L.pic_strerror.restype = C.c_char_p
    L.pic_strerror.argtypes = [_I]
    L.pic_version.restype = C.c_char_p
    L.pic_workspace_size.argtypes = [C.POINTER(Config), C.POINTER(C.c_size_t)]
    L.pic_init.argtypes = [C.POINTER(Config), _P, C.c_size_t, _P, C.POINTER(_P)]
    L.pic_destroy.argtypes = [_P]
    L.pic_destroy.restype = None
    L.pic_load_particles.argtypes = [_P]
    L.pic_step.argtypes = [_P, _I, C.POINTER(StepStats)]
    L.pic_push_deposit.argtypes = [_P, _P, _P, _P, _P, _I, _P, _P]
    L.pic_field_solve.argtypes = [_P, _P, _P, _P, _P, _P, _D, _D, _P, _P, _P, _P]
    L.pic_mcc.argtypes = [_P, C.c_ulonglong, _P, _P]
    L.pic_sort.argtypes = [_P]
    L.pic_diag.argtypes = [_P, C.POINTER(DiagOut)]
    L.pic_diag_average.argtypes = [_P, _I]
    L.pic_diag_get.argtypes = [_P, _I, _P, C.c_size_t, _I]
    L.pic_node_charge.argtypes = [_P, _P]
    L.pic_get_view.argtypes = [_P, C.POINTER(View)]
    L.pic_set_counts.argtypes = [_P, _LL, _LL, C.c_uint32, C.c_uint32, _LL]
    L.pic_mcc_constants.argtypes = [_P, _P, _P, _P, _P]
    L.pic_sort_cells_noalloc.argtypes = [_I, _I, _LL] + [_P] * 16 + [_P, _P]
    L.pic_check_dmul.argtypes = [_P, _P, _P, _LL, _P]
    L.pic_probe_dfma.argtypes = [_I, _I, C.POINTER(_D), C.POINTER(_D)]
    L.pic_substep_histogram.argtypes = [_P, _I, _P]
    L.pic_state_upload.argtypes = [_P, C.POINTER(HostState)]
    L.pic_state_download.argtypes = [_P, C.POINTER(HostState)]
    L.pic_port_field_solve.argtypes = [_P] + [_P] * 8 + [_D, _D] + [_P] * 7
    L.pic_step_host.argtypes = [_P, C.POINTER(HostState), _I, _P]
    L.pic_profile.argtypes = [_P, _I]
    L.pic_profile_read.argtypes = [_P, _P, _P]
    L.pic_cnn_workspace_size.argtypes = [C.POINTER(CnnConfig)]
    L.pic_cnn_workspace_size.restype = C.c_size_t
    L.pic_cnn_init.argtypes = [C.POINTER(CnnConfig), _P, C.c_size_t, _P, C.POINTER(_P)]
    L.pic_cnn_destroy.argtypes = [_P]
    L.pic_cnn_destroy.restype = None
    L.pic_cnn_num_params.argtypes = [_P]
    L.pic_cnn_num_params.restype = _LL
    L.pic_cnn_get_params.argtypes = [_P, _P]
    L.pic_cnn_set_params.argtypes = [_P, _P]
    L.pic_cnn_forward.argtypes = [_P, _P, _I, _P]
    L.pic_cnn_loss_grad.argtypes = [_P, _P, _P, _I, _P, _P]
    L.pic_cnn_train_step.argtypes = [_P, _P, _P, _I, C.c_float, _P]
    L.pic_set_guess.argtypes = [_P, _I, _P]
    L.pic_set_graphs.argtypes = [_P, _I]
    L.pic_set_device_picard.argtypes = [_P, _I]
    L.pic_es_solve.argtypes = [_P, _P, _D, _P, _P]
    L.pic_circuit_get.argtypes = [_P, _P, _P]
    L.pic_circuit_set.argtypes = [_P, _D, _D]
    L.pic_set_drive.argtypes = [_P, _I, _P, _P, _P]
    L.pic_set_picard.argtypes = [_P, _D, _I]
    L.pic_gauss_residual.argtypes = [_P, _P]
    L.pic_save.argtypes = [_P, C.c_char_p]
    L.pic_load.argtypes = [_P, C.c_char_p]
    L.pic_fourier_bessel.argtypes = [_P, _I, _I, _I, _P]
    L.pic_ensemble_create.argtypes = [_P, _I, C.POINTER(_P)]
    L.pic_ensemble_destroy.argtypes = [_P]
    L.pic_ensemble_destroy.restype = None
    L.pic_ensemble_step.argtypes = [_P, _I, _P]
    L.pic_ensemble_set_persistent.argtypes = [_P, _I]
    L.pic_ensemble_tune.argtypes = [_P, _I, C.POINTER(C.c_float), C.POINTER(_I), C.POINTER(_D)]
    L.pic_guess_sample.argtypes = [_P, _P, _P, C.POINTER(_I)]
    return L


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load_lib()
    return _lib


PIC_GUESS_PLAIN, PIC_GUESS_EXTRAP, PIC_GUESS_CNN = 0, 1, 2
PIC_FIELD_EM, PIC_FIELD_ES = 0, 1
CNN_IN, CNN_OUT = 14, 2


class PicError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, lib().pic_strerror(code).decode(), code))


def _check(code, what):
    if code != PIC_OK:
        raise PicError(code, what)
    return code


# ----------------------------------------------------------- named workloads
def small_reactor(**kw):
    """32(r) x 64(z), R = 0.1 m, L = 0.03 m, argon 2 Pa / 300 K, 60 MHz 100 V,
    40k macro-particles per species at 1e15 m^-3, Te = 3 eV, Ti = 0.026 eV,
    dt = 1/(200 f), Picard tolerance 1e-8, seed 0."""
    f = 60e6
    cfg = dict(nr=32, nz=64, R=0.1, L=0.03, dt=1.0 / (200 * f), freq=f, volt=100.0,
               gas_pressure=2.0, gas_temp=300.0, n0=1e15, te_ev=3.0, ti_ev=0.026,
               np_init=40000, capacity_factor=1.5, picard_tol=1e-8, picard_max=50, mcc_on=1,
               bz=0.0, eps=0.0, mu=0.0, seed=0, precision=PIC_FP64, field_model=0, cblock=0.0,
               ions_fixed=0, feed=0, ring_cells=0, eps_ring=1.0, axis_cells=0,
               sigma_ring=0.0, port_cells=0, port_len=0.0, port_rin=0, eps_port=1.0,
               port_grade=1.0)
    cfg.update(kw)
    return cfg


def large_reactor(**kw):
    """256(r) x 384(z), R = 0.3 m, L = 0.03 m, argon 2 Pa / 300 K, 100 MHz 200 V,
    16M macro-particles per species at 1e15 m^-3 (Te = 3 eV, Ti = 0.026 eV),
    dt = 1/(400 f), Picard tolerance 1e-8, seed 1."""
    f = 100e6
    cfg = dict(nr=256, nz=384, R=0.3, L=0.03, dt=1.0 / (400 * f), freq=f, volt=200.0,
               gas_pressure=2.0, gas_temp=300.0, n0=1e15, te_ev=3.0, ti_ev=0.026,
               np_init=16 * 1024 * 1024, capacity_factor=1.25, picard_tol=1e-8, picard_max=50,
               mcc_on=1, bz=0.0, eps=0.0, mu=0.0, seed=1, precision=PIC_FP64, field_model=0,
               cblock=0.0, ions_fixed=0, feed=0, ring_cells=0, eps_ring=1.0, axis_cells=0,
               sigma_ring=0.0, port_cells=0, port_len=0.0, port_rin=0, eps_port=1.0,
               port_grade=1.0)
    cfg.update(kw)
    return cfg


FIELDS = ("cell", "a", "b", "vr", "vt", "vz", "w", "id")


class Pic:
    """One discharge on one GPU.  Owns a torch uint8 workspace on ``device``."""

    def __init__(self, cfg: dict, device="cuda:0", stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.cfg = dict(cfg)
        self._c = Config(**self.cfg)
        nbytes = C.c_size_t(0)
        _check(lib().pic_workspace_size(C.byref(self._c), C.byref(nbytes)), "pic_workspace_size")
        self.ws_bytes = int(nbytes.value)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = _P()
        _check(lib().pic_init(C.byref(self._c), self.ws.data_ptr(), self.ws_bytes,
                              self.stream.cuda_stream, C.byref(h)), "pic_init")
        self._h = h
        self.nr, self.nz = self.cfg["nr"], self.cfg["nz"]

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ methods
    def load_particles(self):
        _check(lib().pic_load_particles(self._h), "pic_load_particles")

    def step(self, n=1, check=True):
        """Advances n steps; returns (status, statistics of the last step).
        check: raise on every error except PIC_E_SUBSTEP, which the library
        reports after completing the step (a particle stopped at the sub-step
        cap, counted in ``substep_err``); the status is returned either way."""
        st = StepStats()
        rc = lib().pic_step(self._h, int(n), C.byref(st))
        if check and rc != PIC_E_SUBSTEP:
            _check(rc, "pic_step")
        return rc, st.as_dict()

    def push_deposit(self, er_half, ez_half, ir, iz, write=False, counters=None, ke_lost=None):
        _check(lib().pic_push_deposit(self._h, er_half.data_ptr(), ez_half.data_ptr(),
                                      ir.data_ptr(), iz.data_ptr(), 1 if write else 0,
                                      counters.data_ptr() if counters is not None else None,
                                      ke_lost.data_ptr() if ke_lost is not None else None),
               "pic_push_deposit")

    def es_solve(self, Q, phi0, er, ez):
        """Electrostatic fields (Eq. 8) of node charges Q (device tensors)."""
        _check(lib().pic_es_solve(self._h, Q.data_ptr(), float(phi0), er.data_ptr(),
                                  ez.data_ptr()), "pic_es_solve")

    def field_solve(self, er0, ez0, h0, ir, iz, v0, v1, er1, ez1, h1, src=None):
        _check(lib().pic_field_solve(self._h, er0.data_ptr(), ez0.data_ptr(), h0.data_ptr(),
                                     ir.data_ptr(), iz.data_ptr(), float(v0), float(v1),
                                     er1.data_ptr(), ez1.data_ptr(), h1.data_ptr(),
                                     src.data_ptr() if src is not None else None),
               "pic_field_solve")

    def port_field_solve(self, er0, ez0, h0, hp0, erp0, ezp0, ir, iz, phi0, phi1, er1, ez1, h1,
                         hp1, erp1, ezp1, src=None):
        """pic_port_field_solve: the field solve with the axial port's fields
        (device tensors in pic_view's port layout)."""
        a = [er0, ez0, h0, hp0, erp0, ezp0, ir, iz]
        b = [er1, ez1, h1, hp1, erp1, ezp1]
        _check(lib().pic_port_field_solve(self._h, *[t.data_ptr() for t in a], float(phi0),
                                          float(phi1), *[t.data_ptr() for t in b],
                                          src.data_ptr() if src is not None else None),
               "pic_port_field_solve")

    def circuit(self):
        """(q^n, phi^n): blocking-capacitor charge and electrode potential."""
        q, phi = _D(0.0), _D(0.0)
        _check(lib().pic_circuit_get(self._h, C.addressof(q), C.addressof(phi)), "pic_circuit_get")
        return q.value, phi.value

    def set_circuit(self, q, phi):
        _check(lib().pic_circuit_set(self._h, float(q), float(phi)), "pic_circuit_set")

    def save(self, path):
        """Checkpoint of the complete state at the current step."""
        _check(lib().pic_save(self._h, os.fsencode(path)), "pic_save")

    def load(self, path):
        """Resume from a checkpoint written by save (same mesh, model, precision)."""
        _check(lib().pic_load(self._h, os.fsencode(path)), "pic_load")

    def set_picard(self, tol, kmax):
        """Picard tolerance and iteration limit of the following steps."""
        _check(lib().pic_set_picard(self._h, float(tol), int(kmax)), "pic_set_picard")

    def set_drive(self, amp=(), freq=(), phase=()):
        """V(t) = sum_k amp[k] sin(2 pi freq[k] t + phase[k]); empty restores the sine."""
        n = len(amp)
        A, Fq, Ph = (_D * max(n, 1))(*amp), (_D * max(n, 1))(*freq), (_D * max(n, 1))(*phase)
        _check(lib().pic_set_drive(self._h, n, C.addressof(A), C.addressof(Fq), C.addressof(Ph)),
               "pic_set_drive")

    def fourier_bessel(self, alpha, row, nmodes, out=None):
        """Fourier-Bessel coefficients (Eq. A2) of E_z (alpha 0) or E_r (alpha 1) at
        one axial row of E^n, into the device tensor ``out`` (allocated if None)."""
        t = self.torch
        if out is None:
            out = t.empty(nmodes, dtype=t.float64, device=self.device)
        _check(lib().pic_fourier_bessel(self._h, int(alpha), int(row), int(nmodes),
                                        out.data_ptr()), "pic_fourier_bessel")
        return out

    def mcc(self, step):
        counts = (_LL * 8)()
        de = _D(0.0)
        rc = lib().pic_mcc(self._h, int(step), C.addressof(counts), C.addressof(de))
        return rc, list(counts), de.value

    def sort(self):
        _check(lib().pic_sort(self._h), "pic_sort")

    def diag(self):
        d = DiagOut()
        _check(lib().pic_diag(self._h, C.byref(d)), "pic_diag")
        return {"kinetic": list(d.kinetic), "field": d.field, "charge": list(d.charge),
                "n": list(d.n)}

    def diag_average(self, enable=True):
        """Start (clearing the averages) or stop the per-step diagnostics
        (pic_diag_average): time-averaged densities and ion fluxes, and the
        continuity residual of each committed step."""
        _check(lib().pic_diag_average(self._h, 1 if enable else 0), "pic_diag_average")

    def diag_get(self, kind):
        """One diagnostic of pic_diag_get as a host numpy array (see
        include/pic.h for the layouts): GAUSS and CONTINUITY (nr+1, nz+1);
        DENSITY_AVG (2, nr+1, nz+1) [m^-3]; ION_FLUX_AVG (2, nr+1) [m^-2 s^-1]
        into z = 0 and z = L; FIELDS (er, ez, h); COUNTS (n_e, n_i, step, steps
        averaged)."""
        nr, nz = self.nr, self.nz
        nn = (nr + 1) * (nz + 1)
        if kind == PIC_DIAG_ENERGY:
            return self.diag()
        shapes = {PIC_DIAG_GAUSS: ((nn,), np.float64), PIC_DIAG_CONTINUITY: ((nn,), np.float64),
                  PIC_DIAG_DENSITY_AVG: ((2 * nn,), np.float64),
                  PIC_DIAG_ION_FLUX_AVG: ((2 * (nr + 1),), np.float64),
                  PIC_DIAG_FIELDS: ((nr * (nz + 1) + (nr + 1) * nz + nr * nz,), np.float64),
                  PIC_DIAG_COUNTS: ((4,), np.int64)}
        shape, dt = shapes[kind]
        out = np.zeros(shape, dtype=dt)
        _check(lib().pic_diag_get(self._h, int(kind), out.ctypes.data, out.nbytes, 0), "pic_diag_get")
        if kind in (PIC_DIAG_GAUSS, PIC_DIAG_CONTINUITY):
            return out.reshape(nr + 1, nz + 1)
        if kind == PIC_DIAG_DENSITY_AVG:
            return out.reshape(2, nr + 1, nz + 1)
        if kind == PIC_DIAG_ION_FLUX_AVG:
            return out.reshape(2, nr + 1)
        if kind == PIC_DIAG_FIELDS:
            a, b = nr * (nz + 1), (nr + 1) * nz
            return out[:a].copy(), out[a:a + b].copy(), out[a + b:].copy()
        return out

    def node_charge(self):
        t = self.torch
        q = t.zeros((self.nr + 1) * (self.nz + 1), dtype=t.float64, device=self.device)
        _check(lib().pic_node_charge(self._h, q.data_ptr()), "pic_node_charge")
        return q

    def gauss_residual(self):
        """eps div_h E - Q on the interior nodes (device tensor, zero elsewhere)."""
        t = self.torch
        r = t.empty((self.nr + 1) * (self.nz + 1), dtype=t.float64, device=self.device)
        _check(lib().pic_gauss_residual(self._h, r.data_ptr()), "pic_gauss_residual")
        return r

    def mcc_constants(self):
        v = [_D(0.0) for _ in range(4)]
        _check(lib().pic_mcc_constants(self._h, *[C.addressof(x) for x in v]), "pic_mcc_constants")
        return tuple(x.value for x in v)

    def profile(self, enable=True):
        _check(lib().pic_profile(self._h, 1 if enable else 0), "pic_profile")

    def profile_read(self):
        ms = _D(0.0)
        nl = _LL(0)
        _check(lib().pic_profile_read(self._h, C.addressof(ms), C.addressof(nl)),
               "pic_profile_read")
        return ms.value, nl.value

    # ---------------------------------------------------------- state views
    def _raw_view(self):
        v = View()
        _check(lib().pic_get_view(self._h, C.byref(v)), "pic_get_view")
        return v

    def _tensor(self, ptr, count, dtype):
        t = self.torch
        itemsize = t.empty((), dtype=dtype).element_size()
        off = ptr - self.ws.data_ptr()
        assert 0 <= off and off + count * itemsize <= self.ws_bytes
        return self.ws[off: off + count * itemsize].view(dtype)

    def view(self):
        """torch views (no copy) of the current particle arrays and fields."""
        t = self.torch
        v = self._raw_view()
        out = {"n": list(v.n), "cap": list(v.cap), "next_id": list(v.next_id), "step": v.step,
               "species": []}
        real = t.float32 if v.real_size == 4 else t.float64
        dt = {"cell": t.int32, "id": t.int32}
        for s in range(2):
            out["species"].append({k: self._tensor(getattr(v, k)[s], v.cap[s],
                                                   dt.get(k, real)) for k in FIELDS})
        out["real_dtype"] = real
        nr, nz = self.nr, self.nz
        out["er"] = self._tensor(v.er, nr * (nz + 1), t.float64)
        out["ez"] = self._tensor(v.ez, (nr + 1) * nz, t.float64)
        out["h"] = self._tensor(v.h, nr * nz, t.float64)
        out["wall"] = self._tensor(v.wall, 2 * (2 * (nr + 1) + nz + 1), t.float64)
        out["qcond"] = self._tensor(v.qcond, (nr + 1) * (nz + 1), t.float64)
        if v.port_m:
            m, q = v.port_m, v.port_cells
            out["port_h"] = self._tensor(v.port_h, m * q, t.float64)
            out["port_er"] = self._tensor(v.port_er, m * q, t.float64)
            out["port_ez"] = self._tensor(v.port_ez, (m + 1) * q, t.float64)
        return out

    def wall_charge(self):
        """Charge absorbed at the walls since pic_init (host copy): per species
        a dict of the z = 0, z = L and r = R node tallies [C]."""
        self.torch.cuda.synchronize(self.device)
        w = self.view()["wall"].cpu().numpy()
        nr, nz = self.nr, self.nz
        blk = 2 * (nr + 1) + nz + 1
        return [{"z0": w[s * blk:s * blk + nr + 1], "zl": w[s * blk + nr + 1:s * blk + 2 * (nr + 1)],
                 "r": w[s * blk + 2 * (nr + 1):(s + 1) * blk]} for s in range(2)]

    def set_state(self, species, er=None, ez=None, h=None, next_ids=None, step=0):
        """Copy host (numpy) species dicts and fields into the context."""
        t = self.torch
        v = self.view()
        ns = []
        for s, sp in enumerate(species):
            n = len(sp["cell"])
            if n > v["cap"][s]:
                raise PicError(PIC_E_STATE, "set_state")
            real = np.float32 if v["real_dtype"] == t.float32 else np.float64
            for k in FIELDS:
                if k == "id":
                    src = np.ascontiguousarray(sp[k]).astype(np.uint32).view(np.int32)
                elif k == "cell":
                    src = np.ascontiguousarray(sp[k], dtype=np.int32)
                else:
                    src = np.ascontiguousarray(sp[k], dtype=real)
                v["species"][s][k][:n].copy_(t.from_numpy(src))
            ns.append(n)
        for name, arr in (("er", er), ("ez", ez), ("h", h)):
            if arr is not None:
                v[name].copy_(t.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)))
        if next_ids is None:
            next_ids = [int(np.max(sp["id"])) + 1 if len(sp["id"]) else 0 for sp in species]
        self.torch.cuda.synchronize(self.device)
        _check(lib().pic_set_counts(self._h, ns[0], ns[1], next_ids[0], next_ids[1], step),
               "pic_set_counts")

    def substep_histogram(self, enable=-1):
        """The 16 bins of accepted sub-steps per particle (pic_substep_histogram)
        as they stand, then enable = 1 clears them and counts from the next
        step, 0 stops counting, -1 leaves the counting as is."""
        h = np.zeros(16, dtype=np.uint64)
        _check(lib().pic_substep_histogram(self._h, int(enable), h.ctypes.data), "pic_substep_histogram")
        return h

    def host_state(self, pinned=True):
        """Host buffers for the whole state (capacity-sized species arrays in
        the context's layout, pinned by default) for state_upload /
        state_download: {"species": [dict of FIELDS tensors] * 2, "er", "ez",
        "h", "n", "next_id", "step"}."""
        t = self.torch
        v = self.view()
        hs = {"species": [{k: t.empty_like(v["species"][s][k], device="cpu").pin_memory()
                           if pinned else t.empty_like(v["species"][s][k], device="cpu")
                           for k in FIELDS} for s in range(2)],
              "n": list(v["cap"]), "next_id": [0, 0], "step": 0}
        for k in ("er", "ez", "h"):
            hs[k] = t.empty_like(v[k], device="cpu").pin_memory() if pinned else \
                t.empty_like(v[k], device="cpu")
        return hs

    def _host_struct(self, hs):
        H = HostState()
        for s in range(2):
            H.n[s] = int(hs["n"][s])
            H.next_id[s] = int(hs["next_id"][s])
            sp = hs["species"][s]
            for k in FIELDS:
                getattr(H, k)[s] = sp[k].data_ptr()
        H.step = int(hs["step"])
        for k in ("er", "ez", "h"):
            setattr(H, k, hs[k].data_ptr() if hs.get(k) is not None else None)
        return H

    def state_upload(self, hs):
        """Host -> device through pic_state_upload (asynchronous on the
        context's stream): the first hs["n"][s] particles of each species, the
        fields given, counts, next ids and step."""
        self._hs_keep = hs  # the host memory stays referenced while copies may run
        _check(lib().pic_state_upload(self._h, C.byref(self._host_struct(hs))), "pic_state_upload")

    def state_download(self, hs):
        """Device -> host through pic_state_download (synchronising): fills the
        buffers of hs and its counts, next ids and step."""
        hs["n"] = [hs["species"][s]["cell"].numel() for s in range(2)]
        H = self._host_struct(hs)
        _check(lib().pic_state_download(self._h, C.byref(H)), "pic_state_download")
        hs["n"] = [H.n[0], H.n[1]]
        hs["next_id"] = [H.next_id[0], H.next_id[1]]
        hs["step"] = H.step
        return hs

    def step_host(self, hs, n=1, check=True):
        """n steps of a state kept in (pinned) host memory through pic_step_host:
        per step host -> device, step, device -> host into the buffers of hs,
        with each step's download overlapped with the next step's upload.
        The host arrays of hs hold the context's capacity (host_state does);
        hs["n"] are the particles in them.  Returns (code, stats of the last
        step) and updates hs's counts."""
        for s in range(2):
            if hs["species"][s]["cell"].numel() < self.view()["cap"][s]:
                raise ValueError("host arrays must hold the context's capacity")
        H = self._host_struct(hs)
        st = StepStats()
        rc = lib().pic_step_host(self._h, C.byref(H), int(n), C.addressof(st))
        if check and rc not in (PIC_OK, PIC_E_SUBSTEP):
            _check(rc, "pic_step_host")
        hs["n"] = [H.n[0], H.n[1]]
        hs["next_id"] = [H.next_id[0], H.next_id[1]]
        hs["step"] = H.step
        return rc, st.as_dict()

    def get_state(self, s):
        v = self.view()
        n = v["n"][s]
        self.torch.cuda.synchronize(self.device)
        out = {k: v["species"][s][k][:n].cpu().numpy().copy() for k in FIELDS}
        out["id"] = out["id"].view(np.uint32)
        return out

    def fields(self):
        v = self.view()
        self.torch.cuda.synchronize(self.device)
        return tuple(v[k].cpu().numpy().copy() for k in ("er", "ez", "h"))


def probe_dfma(blocks_per_sm=4, iters=1 << 16):
    """Measured FP64 FMA throughput (pic_probe_dfma): (seconds, TFLOP/s)."""
    sec, tf = C.c_double(0.0), C.c_double(0.0)
    _check(lib().pic_probe_dfma(int(blocks_per_sm), int(iters), C.byref(sec), C.byref(tf)),
           "pic_probe_dfma")
    return sec.value, tf.value


def check_dmul(x, y):
    """x * y elementwise through the integer-pipe binary64 multiply of the FP64
    mover (pic_check_dmul); x, y: float64 CUDA tensors of one shape."""
    import torch
    x, y = x.contiguous(), y.contiguous()
    out = torch.empty_like(x)
    _check(lib().pic_check_dmul(x.data_ptr(), y.data_ptr(), out.data_ptr(), x.numel(),
                                torch.cuda.current_stream(x.device).cuda_stream), "pic_check_dmul")
    return out


class Cnn:
    """The learned Picard start (include/pic_guess.h): a stack of 3x3
    convolutions on the (nr+1) x (nz+1) grid, BF16 tensor-core kernels with
    FP32 accumulation.  Owns a torch uint8 workspace on ``device``."""

    def __init__(self, nr, nz, depth=5, width=64, batch=8, seed=0, device="cuda:0", stream=None):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        self.nr, self.nz, self.depth, self.width, self.batch = nr, nz, depth, width, batch
        self._c = CnnConfig(nr=nr, nz=nz, width=width, depth=depth, batch=batch, seed=seed)
        nb = lib().pic_cnn_workspace_size(C.byref(self._c))
        if nb == 0:
            raise PicError(PIC_E_CONFIG, "pic_cnn_workspace_size")
        self.ws = torch.empty(int(nb), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = _P()
        _check(lib().pic_cnn_init(C.byref(self._c), self.ws.data_ptr(), int(nb),
                                  self.stream.cuda_stream, C.byref(h)), "pic_cnn_init")
        self._h = h
        self.num_params = int(lib().pic_cnn_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        return (self.nr + 1, self.nz + 1)

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params, dtype=np.float32)
        _check(lib().pic_cnn_get_params(self._h, out.ctypes.data), "pic_cnn_get_params")
        return out

    def set_params(self, v):
        import numpy as np
        v = np.ascontiguousarray(v, dtype=np.float32)
        assert v.size == self.num_params
        _check(lib().pic_cnn_set_params(self._h, v.ctypes.data), "pic_cnn_set_params")

    def forward(self, x):
        """x: float32 device tensor [B, 14, nr+1, nz+1] -> [B, 2, nr+1, nz+1]."""
        x = x.contiguous()
        y = self.torch.empty((x.shape[0], CNN_OUT) + self.shape, dtype=self.torch.float32,
                             device=self.device)
        _check(lib().pic_cnn_forward(self._h, x.data_ptr(), int(x.shape[0]), y.data_ptr()),
               "pic_cnn_forward")
        return y

    def loss_grad(self, x, t, grad=True):
        import numpy as np
        x, t = x.contiguous(), t.contiguous()
        loss = C.c_double(0.0)
        g = np.empty(self.num_params, dtype=np.float32) if grad else None
        _check(lib().pic_cnn_loss_grad(self._h, x.data_ptr(), t.data_ptr(), int(x.shape[0]),
                                       C.byref(loss), g.ctypes.data if grad else None),
               "pic_cnn_loss_grad")
        return loss.value, g

    def train_step(self, x, t, lr):
        x, t = x.contiguous(), t.contiguous()
        loss = C.c_double(0.0)
        _check(lib().pic_cnn_train_step(self._h, x.data_ptr(), t.data_ptr(), int(x.shape[0]),
                                        float(lr), C.byref(loss)), "pic_cnn_train_step")
        return loss.value


def set_guess(pic, mode, cnn=None):
    """Picard start of the following steps of ``pic`` (PIC_GUESS_*)."""
    _check(lib().pic_set_guess(pic._h, int(mode), cnn._h if cnn is not None else None),
           "pic_set_guess")


def guess_sample(pic):
    """(inputs [14, nr+1, nz+1], target [2, nr+1, nz+1]) of the last step, or None."""
    import torch
    H, W = pic.nr + 1, pic.nz + 1
    x = torch.empty((CNN_IN, H, W), dtype=torch.float32, device=pic.device)
    t = torch.empty((CNN_OUT, H, W), dtype=torch.float32, device=pic.device)
    valid = _I(0)
    _check(lib().pic_guess_sample(pic._h, x.data_ptr(), t.data_ptr(), C.byref(valid)),
           "pic_guess_sample")
    return (x, t) if valid.value else None


def set_graphs(pic, on=True):
    """Replay the Picard passes of ``pic`` from captured CUDA graphs."""
    _check(lib().pic_set_graphs(pic._h, 1 if on else 0), "pic_set_graphs")


def set_device_picard(pic, on=True):
    """Run the Picard iteration as one conditional graph per step (graphs on,
    timing off; the default) or from the host, one wait per pass."""
    _check(lib().pic_set_device_picard(pic._h, 1 if on else 0), "pic_set_device_picard")


class Ensemble:
    """Independent discharges (``Pic`` members, each on its own stream) stepped
    side by side (include/pic_ensemble.h).  Does not own the members."""

    def __init__(self, members):
        self.members = list(members)
        arr = (_P * len(self.members))(*[m._h for m in self.members])
        h = _P()
        _check(lib().pic_ensemble_create(arr, len(self.members), C.byref(h)),
               "pic_ensemble_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().pic_ensemble_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1, check=True):
        st = (StepStats * len(self.members))()
        rc = lib().pic_ensemble_step(self._h, int(n), st)
        if check and rc != PIC_E_SUBSTEP:  # non-fatal, as in Pic.step
            _check(rc, "pic_ensemble_step")
        return rc, [s.as_dict() for s in st]

    def set_persistent(self, on=True):
        """Persistent rounds (one push launch per species over all members) or
        per-member rounds (each member's pass replayed from its CUDA graph)."""
        _check(lib().pic_ensemble_set_persistent(self._h, int(bool(on))),
               "pic_ensemble_set_persistent")

    def tune(self, rounds=3):
        """(grid fraction, persistent?, best ms per round of the 6 candidates:
        per-member rounds at fractions 1, 1/2, 1/4, then persistent ones; -1
        where the members do not allow persistent rounds)."""
        f = C.c_float(0.0)
        pers = _I(0)
        ms = (_D * 6)()
        _check(lib().pic_ensemble_tune(self._h, int(rounds), C.byref(f), C.byref(pers), ms),
               "pic_ensemble_tune")
        return float(f.value), bool(pers.value), list(ms)
