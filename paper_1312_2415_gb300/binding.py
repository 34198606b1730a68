"""ctypes binding of libdmrg_gb300.so (argument marshalling only).

Every call goes straight to the C ABI declared in include/dmrg_gb300.h; the numeric
work runs in the library's CUDA kernels.  Import fails loudly when the compiled
library is missing: there is no other implementation to fall back to.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_LIB = os.path.join(_HERE, "_build", "libdmrg_gb300.so")

OK, EINVAL, ESYMM, ENOTCONV, ENOMEM, ECUDA, EINTERNAL = 0, -1, -2, -3, -4, -5, -6
GROUP_ORDER = [1, 2, 2, 2, 4, 4, 4, 8]


class DMRGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dmrg error {code}: {msg}")
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [
        ("matvecs", ctypes.c_int64), ("davidson_iters", ctypes.c_int64),
        ("micro_iters", ctypes.c_int64), ("matvec_flops", ctypes.c_double),
        ("last_matvec_flops", ctypes.c_double), ("last_matvec_tasks", ctypes.c_int64),
        ("t_update_ms", ctypes.c_double), ("t_trunc_ms", ctypes.c_double),
        ("t_plan_ms", ctypes.c_double), ("t_total_ms", ctypes.c_double),
        ("last_w_disc", ctypes.c_double), ("max_w_disc", ctypes.c_double),
        ("k_phase1_ms", ctypes.c_double), ("k_phase2_ms", ctypes.c_double),
        ("k_launches", ctypes.c_int64), ("k_phase1_flops", ctypes.c_double),
        ("k_phase2_flops", ctypes.c_double), ("kernels_launched", ctypes.c_int64),
        ("tc_matvecs", ctypes.c_int64), ("tc_flops", ctypes.c_double),
        ("tc_phase1_ms", ctypes.c_double), ("tc_phase2_ms", ctypes.c_double),
        ("tc_phase1_flops", ctypes.c_double), ("tc_phase2_flops", ctypes.c_double),
        ("tc_phase1_bytes", ctypes.c_double), ("tc_phase2_bytes", ctypes.c_double),
        ("rdm_passes", ctypes.c_int64), ("rdm_ms", ctypes.c_double), ("rdm_flops", ctypes.c_double),
    ]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_I64 = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "dmrg_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, _I, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "dmrg_set_integrals": (ctypes.c_int, [_P, ctypes.c_double, _D, _D]),
    "dmrg_set_schedule": (ctypes.c_int, [_P, ctypes.c_int, _I, _D, _I, _D, ctypes.c_double, ctypes.c_int]),
    "dmrg_init_mps": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "dmrg_set_precision": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "dmrg_get_mps": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "dmrg_set_mps": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_size_t]),
    "dmrg_solve": (ctypes.c_int, [_P, _D, _D]),
    "dmrg_canonicalize": (ctypes.c_int, [_P, ctypes.c_int]),
    "dmrg_two_site_layout": (ctypes.c_int, [_P, ctypes.c_int, _I64, _I, _I64]),
    "dmrg_tt_to_x": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "dmrg_heff_matvec": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "dmrg_heff_diag": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]),
    "dmrg_rdm": (ctypes.c_int, [_P, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "dmrg_push_excitation": (ctypes.c_int, [_P, ctypes.c_double]),
    "dmrg_clear_excitations": (ctypes.c_int, [_P]),
    "dmrg_excitation_count": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "dmrg_heff_matvec_noalloc": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_size_t]),
    "dmrg_davidson": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, _D, _I]),
    "dmrg_truncate": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_size_t, _D]),
    "dmrg_set_next_site": (ctypes.c_int, [_P, ctypes.c_int]),
    "dmrg_update_operators": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "dmrg_sweep_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                       _D, _D, _I]),
    "dmrg_solve_history": (ctypes.c_int, [_P, _I, _I, _D, _D]),
    "dmrg_extrapolate": (ctypes.c_int, [_D, _D, ctypes.c_int, _D, _D]),
    "dmrg_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.POINTER(_P), _I, ctypes.c_int,
                                         ctypes.c_int]),
    "dmrg_batch_io": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                     ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)]),
    "dmrg_batch_run": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.c_size_t]),
    "dmrg_batch_info": (ctypes.c_int, [_P, _D, _I, _I, _D, _D]),
    "dmrg_energy": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_void_p, _D, ctypes.c_size_t]),
    "dmrg_batch_davidson": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_void_p), ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, _D, _I, _I, ctypes.c_size_t]),
    "dmrg_batch_last_error": (ctypes.c_char_p, [_P]),
    "dmrg_batch_destroy": (None, [_P]),
    "dmrg_test_tc_timeout": (ctypes.c_int, [ctypes.c_int]),
    "dmrg_set_device_memory_cap": (ctypes.c_int, [ctypes.c_size_t]),
    "dmrg_device_memory_in_use": (ctypes.c_int, [ctypes.POINTER(ctypes.c_size_t)]),
    "dmrg_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "dmrg_last_error": (ctypes.c_char_p, [_P]),
    "dmrg_destroy": (None, [_P]),
}

EXPORTED = sorted(_SIGS)
_libs = {}


def load(path=None):
    """Load (once) the compiled library; raises OSError when it is absent."""
    path = os.path.abspath(path or os.environ.get("DMRG_GB300_LIB", DEFAULT_LIB))
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise OSError(f"{path} not built: run __graft_entry__.build() (nvcc, sm_103a)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _libs[path] = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(_D)


def _ptr_and_stream(arr):
    """(pointer, stream): numpy arrays are host buffers (stream 0); torch CUDA tensors
    are passed as device pointers on the current torch stream."""
    if isinstance(arr, np.ndarray):
        assert arr.dtype == np.float64 and arr.flags.c_contiguous
        return arr.ctypes.data, 0
    import torch  # device memory / streams only
    assert arr.is_cuda and arr.dtype == torch.float64 and arr.is_contiguous()
    s = torch.cuda.current_stream(arr.device).cuda_stream
    return arr.data_ptr(), (s if s else _default_stream_handle(arr.device))


def _default_stream_handle(device):
    # the legacy default stream is handle 0, which the ABI reserves for host
    # pointers; cudaStreamLegacy (0x1) names the same stream
    return 1


class Context:
    """One DMRG problem on the current GPU (mirrors the dmrg_* calls)."""

    def __init__(self, L, orb_irrep, N, two_S, target_irrep, group=None, precision=0, lib=None):
        self.lib = load(lib)
        if group is None:
            n_ir = max(orb_irrep + [target_irrep]) + 1
            group = {1: 0, 2: 1, 3: 4, 4: 4}.get(n_ir, 7)
        self.L = L
        ir = (ctypes.c_int * L)(*orb_irrep)
        h = _P()
        self._check(self.lib.dmrg_create(ctypes.byref(h), L, group, ir, N, two_S, target_irrep, precision), None)
        self.h = h

    def _check(self, rc, h="self"):
        if rc != OK:
            msg = self.lib.dmrg_last_error(self.h if h == "self" else None)
            raise DMRGError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_integrals(self, h, V, econst=0.0):
        h = np.ascontiguousarray(h, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        self._check(self.lib.dmrg_set_integrals(self.h, float(econst), _dptr(h), _dptr(V)))

    def set_schedule(self, D, e_conv, n_max, noise, davidson_tol=1e-10, davidson_max_iter=100):
        n = len(D)
        Da = (ctypes.c_int * n)(*D)
        Ea = np.ascontiguousarray(e_conv, dtype=np.float64)
        Na = (ctypes.c_int * n)(*n_max)
        Za = np.ascontiguousarray(noise, dtype=np.float64)
        self._check(self.lib.dmrg_set_schedule(self.h, n, Da, _dptr(Ea), Na, _dptr(Za),
                                               float(davidson_tol), int(davidson_max_iter)))

    def solve_history(self):
        """(D, energy, w_disc) per schedule instruction of the last solve (Sec. 4.3)."""
        n = ctypes.c_int(0)
        self._check(self.lib.dmrg_solve_history(self.h, ctypes.byref(n), None, None, None))
        D = np.zeros(n.value, dtype=np.int32)
        E, W = np.zeros(n.value), np.zeros(n.value)
        self._check(self.lib.dmrg_solve_history(self.h, ctypes.byref(n), D.ctypes.data_as(_I), _dptr(E),
                                                _dptr(W)))
        return D, E, W

    def set_precision(self, precision, fp64_iters=0):
        self._check(self.lib.dmrg_set_precision(self.h, int(precision), int(fp64_iters)))

    def init_mps(self, seed):
        self._check(self.lib.dmrg_init_mps(self.h, int(seed)))

    def get_mps(self):
        n = ctypes.c_size_t(0)
        self._check(self.lib.dmrg_get_mps(self.h, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        self._check(self.lib.dmrg_get_mps(self.h, buf, ctypes.byref(n)))
        return buf.raw[: n.value]

    def set_mps(self, data):
        self._check(self.lib.dmrg_set_mps(self.h, data, len(data)))

    def canonicalize(self, center):
        self._check(self.lib.dmrg_canonicalize(self.h, int(center)))

    def solve(self):
        em, el = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.dmrg_solve(self.h, ctypes.byref(em), ctypes.byref(el)))
        return em.value, el.value

    def layout(self, site):
        n, nb = ctypes.c_int64(), ctypes.c_int()
        self._check(self.lib.dmrg_two_site_layout(self.h, site, ctypes.byref(n), ctypes.byref(nb), None))
        t = np.zeros((nb.value, 12), dtype=np.int64)
        self._check(self.lib.dmrg_two_site_layout(self.h, site, ctypes.byref(n), ctypes.byref(nb),
                                                  t.ctypes.data_as(_I64)))
        return n.value, t

    def tt_to_x(self, site, out=None):
        if out is None:
            out = np.zeros(self.layout(site)[0])
        p, s = _ptr_and_stream(out)
        self._check(self.lib.dmrg_tt_to_x(self.h, site, p, s))
        return out

    def matvec(self, site, x, y=None):
        if y is None:
            y = np.zeros_like(x)
        px, s = _ptr_and_stream(x)
        py, _ = _ptr_and_stream(y)
        self._check(self.lib.dmrg_heff_matvec(self.h, site, px, py, s))
        return y

    def energy(self, site, x):
        """x^T H_eff x / x^T x in FP64 (dmrg_energy); x: numpy array or CUDA tensor."""
        p, s = _ptr_and_stream(x)
        e = ctypes.c_double()
        self._check(self.lib.dmrg_energy(self.h, site, p, ctypes.byref(e), s))
        return e.value

    def matvec_noalloc(self, site, x, y, stream=0):
        """y = H_eff x without any allocation (x, y: device addresses; see the header)."""
        self._check(self.lib.dmrg_heff_matvec_noalloc(self.h, int(site), int(x), int(y), int(stream)))

    def diag(self, site, out=None):
        if out is None:
            out = np.zeros(self.layout(site)[0])
        p, s = _ptr_and_stream(out)
        self._check(self.lib.dmrg_heff_diag(self.h, site, p, s))
        return out

    def rdm(self, gamma=None, Gamma=None):
        """Spin-summed 1- and 2-RDMs of the current MPS (dmrg_rdm): gamma (L, L) and
        Gamma (L, L, L, L), numpy (host) or float64 CUDA tensors (device)."""
        L = self.L
        if gamma is None:
            gamma, Gamma = np.zeros((L, L)), np.zeros((L,) * 4)
        p1, s = _ptr_and_stream(gamma)
        p2, _ = _ptr_and_stream(Gamma)
        assert gamma.shape == (L, L) and Gamma.shape == (L,) * 4
        self._check(self.lib.dmrg_rdm(self.h, p1, p2, s))
        return gamma, Gamma

    def push_excitation(self, eta):
        """Store the current MPS as the next lower state with weight eta (Sec. 4.3)."""
        self._check(self.lib.dmrg_push_excitation(self.h, float(eta)))

    def clear_excitations(self):
        self._check(self.lib.dmrg_clear_excitations(self.h))

    def excitation_count(self):
        n = ctypes.c_int()
        self._check(self.lib.dmrg_excitation_count(self.h, ctypes.byref(n)))
        return n.value

    def davidson(self, site, x):
        p, s = _ptr_and_stream(x)
        e, it = ctypes.c_double(), ctypes.c_int()
        rc = self.lib.dmrg_davidson(self.h, site, p, s, ctypes.byref(e), ctypes.byref(it))
        if rc not in (OK, ENOTCONV):
            self._check(rc)
        return e.value, it.value, rc == OK

    def truncate(self, site, direction, D, x, noise=0.0):
        p, s = _ptr_and_stream(x)
        w = ctypes.c_double()
        self._check(self.lib.dmrg_truncate(self.h, site, int(direction), int(D), float(noise), p, s,
                                           ctypes.byref(w)))
        return w.value

    def set_next_site(self, site):
        """Hint: the site of the next sweep_step (-1 = unknown); see the header."""
        self._check(self.lib.dmrg_set_next_site(self.h, int(site)))

    def update_operators(self, site, direction):
        """The operator update of a sweep step (after truncate in the same direction)."""
        self._check(self.lib.dmrg_update_operators(self.h, int(site), int(direction)))

    def sweep_step(self, site, direction, D, gamma=0.0):
        e, w, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        rc = self.lib.dmrg_sweep_step(self.h, int(site), int(direction), int(D), float(gamma),
                                      ctypes.byref(e), ctypes.byref(w), ctypes.byref(it))
        if rc not in (OK, ENOTCONV):
            self._check(rc)
        return e.value, w.value, it.value, rc == OK

    def stats(self):
        st = Stats()
        self._check(self.lib.dmrg_stats(self.h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}


def set_device_memory_cap(nbytes, path=None):
    """Cap on the device memory the library holds (0 = none); see the header."""
    rc = load(path).dmrg_set_device_memory_cap(int(nbytes))
    if rc != OK:
        raise DMRGError(rc, "dmrg_set_device_memory_cap")


def test_tc_timeout(on, path=None):
    """Failure-detection test hook: the tensor-core kernel's waits give up (see header)."""
    rc = load(path).dmrg_test_tc_timeout(int(on))
    if rc != OK:
        raise DMRGError(rc, "dmrg_test_tc_timeout")


def device_memory_in_use(path=None):
    n = ctypes.c_size_t(0)
    rc = load(path).dmrg_device_memory_in_use(ctypes.byref(n))
    if rc != OK:
        raise DMRGError(rc, "dmrg_device_memory_in_use")
    return n.value


def extrapolate(w_disc, energy, path=None):
    """Eq. 16: least-squares E(D) = E_exact + C1 w_disc(D); returns (E_exact, C1)."""
    lib = load(path)
    w = np.ascontiguousarray(w_disc, dtype=np.float64)
    e = np.ascontiguousarray(energy, dtype=np.float64)
    e0, c1 = ctypes.c_double(), ctypes.c_double()
    rc = lib.dmrg_extrapolate(_dptr(w), _dptr(e), int(w.size), ctypes.byref(e0), ctypes.byref(c1))
    if rc != OK:
        raise DMRGError(rc, "extrapolate: need two or more points with different discarded weights")
    return e0.value, c1.value


class Batch:
    """Batched mixed-precision matvecs of several contexts (dmrg_batch_*): one grouped
    launch per phase over all instances, replayed from a CUDA graph."""

    def __init__(self, contexts, sites, autotune=True):
        self.contexts = list(contexts)
        self.lib = self.contexts[0].lib
        n = len(self.contexts)
        arr = (_P * n)(*[c.h for c in self.contexts])
        st = (ctypes.c_int * n)(*[int(s) for s in sites])
        h = _P()
        rc = self.lib.dmrg_batch_create(ctypes.byref(h), arr, st, n, int(bool(autotune)))
        if rc != OK:
            raise DMRGError(rc, self.lib.dmrg_last_error(self.contexts[0].h).decode())
        self.h = h

    def io(self, i):
        """(x pointer, y pointer, n) of instance i: the batch's device buffers."""
        x, y, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
        rc = self.lib.dmrg_batch_io(self.h, int(i), ctypes.byref(x), ctypes.byref(y), ctypes.byref(n))
        if rc != OK:
            raise DMRGError(rc, "batch io")
        return x.value, y.value, n.value

    def run(self, xs=None, ys=None):
        """Queue y_i = H_eff x_i for all instances on the current torch stream; xs / ys:
        lists of float64 CUDA tensors (or None for the batch's own buffers)."""
        import torch  # device memory / streams only
        n = len(self.contexts)
        xp = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in (xs or [None] * n)])
        yp = (ctypes.c_void_p * n)(*[(t.data_ptr() if t is not None else None) for t in (ys or [None] * n)])
        s = torch.cuda.current_stream().cuda_stream or _default_stream_handle(None)
        rc = self.lib.dmrg_batch_run(self.h, xp, yp, s)
        if rc != OK:
            raise DMRGError(rc, self.lib.dmrg_batch_last_error(self.h).decode())

    def davidson(self, xs, tol=1e-5, max_iter=100, fp64_energy=True):
        """Davidson for every instance in lockstep (dmrg_batch_davidson) on the current torch
        stream; xs: list of float64 CUDA tensors (start vectors, overwritten by the Ritz
        vectors).  Returns (energies, iterations, converged) as numpy arrays."""
        import torch  # device memory / streams only
        n = len(self.contexts)
        xp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in xs])
        e = np.zeros(n)
        it = np.zeros(n, dtype=np.int32)
        cv = np.zeros(n, dtype=np.int32)
        s = torch.cuda.current_stream().cuda_stream or _default_stream_handle(None)
        rc = self.lib.dmrg_batch_davidson(self.h, xp, float(tol), int(max_iter), int(bool(fp64_energy)),
                                          _dptr(e), it.ctypes.data_as(_I), cv.ctypes.data_as(_I), s)
        if rc not in (OK, ENOTCONV):
            raise DMRGError(rc, self.lib.dmrg_batch_last_error(self.h).decode())
        return e, it, cv.astype(bool)

    def info(self):
        f, ms, tms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        ppu, tpu = ctypes.c_int(), ctypes.c_int()
        self.lib.dmrg_batch_info(self.h, ctypes.byref(f), ctypes.byref(ppu), ctypes.byref(tpu), ctypes.byref(ms),
                                 ctypes.byref(tms))
        return {"flops": f.value, "row_tile": ppu.value, "x_chunk": tpu.value,
                "launch_ms": ms.value, "tune_ms": tms.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.dmrg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

