"""ctypes binding of libtsbz (include/tsbz.h): argument marshalling only.

Every step of the propagation runs inside the library's CUDA kernels.  If
the shared library has not been built this module raises at import time of
``load()``; there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtsbz.so")

TSBZ_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ENONFINITE", -6: "ESTATE"}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_tc": 2}
HXC_SCF, HXC_FROZEN = 0, 1


class TsbzError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"tsbz error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class CellDesc(ctypes.Structure):
    _fields_ = [
        ("a", ctypes.c_double * 3),
        ("n", ctypes.c_int * 3),
        ("n_atoms", ctypes.c_int),
        ("atom_frac", ctypes.POINTER(ctypes.c_double)),
        ("z_ion", ctypes.c_double),
        ("r_erf", ctypes.c_double),
        ("c_core", ctypes.c_double),
        ("sigma_core", ctypes.c_double),
        ("r_proj", ctypes.c_double),
        ("proj_half", ctypes.c_double),
        ("e_kb_s", ctypes.c_double),
        ("e_kb_p", ctypes.c_double),
        ("use_projectors", ctypes.c_int),
        ("n_bands", ctypes.c_int),
        ("occ", ctypes.c_double),
        ("fd_nd", ctypes.c_int),
        ("hxc_mode", ctypes.c_int),
        ("xc", ctypes.c_int),
        ("hartree", ctypes.c_int),
    ]


class Alloc(ctypes.Structure):
    _fields_ = [
        ("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)),
        ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)),
        ("user", ctypes.c_void_p),
    ]


_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_SIGS = {
    "tsbz_version": ([], ctypes.c_int),
    "tsbz_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                     ctypes.POINTER(Alloc)], ctypes.c_int),
    "tsbz_init_cell": ([ctypes.c_void_p, ctypes.POINTER(CellDesc), _I], ctypes.c_int),
    "tsbz_add_subsim": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, ctypes.c_double, ctypes.c_int, _I],
                        ctypes.c_int),
    "tsbz_load_ground_state": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, _D],
                               ctypes.c_int),
    "tsbz_set_kick": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _D], ctypes.c_int),
    "tsbz_set_field": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D], ctypes.c_int),
    "tsbz_propagate": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "tsbz_get_current": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D], ctypes.c_int),
    "tsbz_get_current_stats": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _D, _D], ctypes.c_int),
    "tsbz_get_density": ([ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_size_t], ctypes.c_int),
    "tsbz_get_norms": ([ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_size_t], ctypes.c_int),
    "tsbz_get_step": ([ctypes.c_void_p, ctypes.c_int, _I], ctypes.c_int),
    "tsbz_get_state": ([ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_size_t, _I], ctypes.c_int),
    "tsbz_load_state": ([ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_size_t, ctypes.c_int], ctypes.c_int),
    "tsbz_get_cell_tables": ([ctypes.c_void_p, ctypes.c_int, _D, ctypes.c_size_t, _D, ctypes.c_size_t],
                             ctypes.c_int),
    "tsbz_get_launch_count": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)], ctypes.c_int),
    "tsbz_get_timings": ([ctypes.c_void_p, _D, ctypes.c_int], ctypes.c_int),
    "tsbz_set_profiling": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "tsbz_set_graphs": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "tsbz_set_propagator": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "tsbz_ground_state": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_double, _I, _D],
                          ctypes.c_int),
    "tsbz_autotune": ([ctypes.c_void_p, ctypes.c_int, _I], ctypes.c_int),
    "tsbz_get_variant": ([ctypes.c_void_p, ctypes.c_int, _I, _I, _D, ctypes.c_int], ctypes.c_int),
    "tsbz_set_variant": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "tsbz_selftest_bounded_wait": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _I], ctypes.c_int),
    "tsbz_probe_alu_peak": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D], ctypes.c_int),
    "tsbz_selftest_umma": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _I], ctypes.c_int),
    "tsbz_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "tsbz_destroy": ([ctypes.c_void_p], None),
    "tsbz_shifted_kpoints": ([_D, _I, _D, _D, ctypes.c_size_t], ctypes.c_int),
    "tsbz_halton": ([ctypes.c_int, _D, ctypes.c_size_t], ctypes.c_int),
    "tsbz_pulse_samples": ([ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, ctypes.c_double, ctypes.c_int,
                            _D, ctypes.c_size_t], ctypes.c_int),
    "tsbz_density_noalloc": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _I, ctypes.c_double, ctypes.c_void_p,
                              ctypes.c_void_p], ctypes.c_int),
}


def load(path: str | None = None):
    """Load libtsbz.so (built by ``paper_2112_00920_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libtsbz.so not found at {p}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`; no CPU fallback exists")
    lib = ctypes.CDLL(p)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(_D)


def shifted_kpoints(a, mp, shift) -> np.ndarray:
    """k-points (n, 3) of the shifted Monkhorst-Pack grid (Eq. 10)."""
    lib = load()
    n = int(mp[0] * mp[1] * mp[2])
    out = np.zeros((n, 3))
    aa = np.ascontiguousarray(a, dtype=np.float64)
    mm = (ctypes.c_int * 3)(*[int(v) for v in mp])
    ss = np.ascontiguousarray(shift, dtype=np.float64)
    rc = lib.tsbz_shifted_kpoints(_dptr(aa), mm, _dptr(ss), _dptr(out), out.size)
    if rc:
        raise TsbzError(rc, "tsbz_shifted_kpoints")
    return out


def halton(n: int) -> np.ndarray:
    lib = load()
    out = np.zeros((n, 3))
    rc = lib.tsbz_halton(int(n), _dptr(out), out.size)
    if rc:
        raise TsbzError(rc, "tsbz_halton")
    return out


def pulse_samples(e0, omega0, t_pulse, direction, dt, n_steps) -> np.ndarray:
    lib = load()
    out = np.zeros((2 * n_steps + 1, 3))
    d = np.ascontiguousarray(direction, dtype=np.float64)
    rc = lib.tsbz_pulse_samples(e0, omega0, t_pulse, _dptr(d), dt, int(n_steps), _dptr(out), out.size)
    if rc:
        raise TsbzError(rc, "tsbz_pulse_samples")
    return out


def selftest_bounded_wait(device: int = 0, polls: int = 1000, deliver: bool = False):
    """Run the bounded-wait self-test; returns (return code, kernel status word)."""
    st = ctypes.c_int()
    rc = load().tsbz_selftest_bounded_wait(int(device), int(polls), 1 if deliver else 0, ctypes.byref(st))
    return rc, st.value


def probe_alu_peak(device: int, kind: str, iters: int = 20000):
    """Peak FMA throughput of the device (tsbz_probe_alu_peak): kind "ffma"
    (FP32), "ffma2" (packed FP32x2) or "dfma" (FP64).  Returns (flop/s, ms)."""
    lib = load()
    k = {"ffma": 0, "ffma2": 1, "dfma": 2}[kind]
    f, ms = ctypes.c_double(), ctypes.c_double()
    rc = lib.tsbz_probe_alu_peak(int(device), k, int(iters), ctypes.byref(f), ctypes.byref(ms))
    if rc:
        raise TsbzError(rc, "tsbz_probe_alu_peak")
    return f.value, ms.value


def selftest_umma(device: int, a: np.ndarray, b: np.ndarray, swap_lbo_sbo: bool = False):
    """D = A B^T (128 x 32, K = 16) through the library's tcgen05 building
    blocks (tsbz_selftest_umma).  Returns (status code, status word, D)."""
    fp = ctypes.POINTER(ctypes.c_float)
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = np.ascontiguousarray(b, dtype=np.float32)
    assert a.shape == (128, 16) and b.shape == (32, 16)
    d = np.zeros((128, 32), dtype=np.float32)
    st = ctypes.c_int()
    rc = load().tsbz_selftest_umma(int(device), 1 if swap_lbo_sbo else 0, a.ctypes.data_as(fp), b.ctypes.data_as(fp),
                                   d.ctypes.data_as(fp), ctypes.byref(st))
    return rc, st.value, d


def density_noalloc(psi, occ, rho=None, stream=None):
    """rho(r) = (1/n_k) sum_k sum_b occ |u(r)|^2 of a complex128 CUDA tensor
    psi (n_k, n_b, n3, n2, n1), through tsbz_density_noalloc: the library
    allocates nothing (the result goes to ``rho``, allocated here by torch if
    not given).  Queued on the current torch stream."""
    import torch

    lib = load()
    assert psi.is_cuda and psi.dtype == torch.complex128 and psi.is_contiguous() and psi.dim() == 5
    n_k, n_b, n3, n2, n1 = psi.shape
    if rho is None:
        rho = torch.empty((n3, n2, n1), dtype=torch.float64, device=psi.device)
    assert rho.device == psi.device and rho.dtype == torch.float64 and rho.is_contiguous()
    assert rho.numel() == n3 * n2 * n1
    # the library looks up its static buffer on the current device: make it psi's
    with torch.cuda.device(psi.device):
        if stream is None:
            stream = torch.cuda.current_stream(psi.device).cuda_stream
        nn = (ctypes.c_int * 3)(n1, n2, n3)
        rc = lib.tsbz_density_noalloc(ctypes.c_void_p(psi.data_ptr()), n_k, n_b, nn, float(occ),
                                      ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(stream))
    if rc:
        raise TsbzError(rc, "tsbz_density_noalloc")
    return rho


class Propagator:
    """One library context (tsbz_ctx) on one GPU.

    Device memory comes from torch's caching allocator through the C
    allocator callback; work runs on the current torch CUDA stream unless a
    stream handle is given."""

    def __init__(self, precision: str = "fp64", device: int = 0, stream=None, torch_alloc: bool = True):
        import torch

        self.lib = load()
        self._torch = torch
        self._blocks = {}
        self._alloc_struct = None
        if torch_alloc:
            dev = torch.device("cuda", device)

            @ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
            def _alloc(nbytes, user):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=dev)
                self._blocks[t.data_ptr()] = t
                return t.data_ptr()

            @ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)
            def _free(ptr, user):
                self._blocks.pop(ptr, None)

            self._cb = (_alloc, _free)
            self._alloc_struct = Alloc(_alloc, _free, None)
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.stream = stream
        ctx = ctypes.c_void_p()
        rc = self.lib.tsbz_create(ctypes.byref(ctx), device, PRECISIONS[precision], ctypes.c_void_p(stream),
                                  ctypes.byref(self._alloc_struct) if self._alloc_struct else None)
        if rc:
            raise TsbzError(rc, "tsbz_create failed")
        self.ctx = ctx
        self.precision = precision
        self.cells = []
        self.subs = []

    # -- helpers -------------------------------------------------------------
    def _check(self, rc, what):
        if rc:
            msg = self.lib.tsbz_last_error(self.ctx)
            raise TsbzError(rc, f"{what}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.tsbz_destroy(self.ctx)
            self.ctx = None
            self._blocks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up --------------------------------------------------------------
    def add_cell(self, a, n, atom_frac, n_bands, e_kb_s, e_kb_p, z_ion=4.0, r_erf=0.8, c_core=10.0,
                 sigma_core=1.0, r_proj=1.0, proj_half=8.0, use_projectors=True, occ=2.0, fd_nd=4,
                 hxc="scf", xc=True, hartree=True) -> int:
        fr = np.ascontiguousarray(np.asarray(atom_frac, dtype=np.float64).reshape(-1))
        d = CellDesc()
        d.a[:] = [float(v) for v in a]
        d.n[:] = [int(v) for v in n]
        d.n_atoms = fr.size // 3
        d.atom_frac = _dptr(fr) if fr.size else None
        d.z_ion, d.r_erf, d.c_core, d.sigma_core = z_ion, r_erf, c_core, sigma_core
        d.r_proj, d.proj_half, d.e_kb_s, d.e_kb_p = r_proj, proj_half, e_kb_s, e_kb_p
        d.use_projectors = 1 if (use_projectors and d.n_atoms) else 0
        d.n_bands = int(n_bands)
        d.occ = occ
        d.fd_nd = int(fd_nd)
        d.hxc_mode = HXC_FROZEN if hxc == "frozen" else HXC_SCF
        d.xc = 1 if xc else 0
        d.hartree = 1 if hartree else 0
        cid = ctypes.c_int()
        self._check(self.lib.tsbz_init_cell(self.ctx, ctypes.byref(d), ctypes.byref(cid)), "tsbz_init_cell")
        self.cells.append(dict(n=tuple(int(v) for v in n), n_bands=int(n_bands), n_atoms=d.n_atoms))
        return cid.value

    def add_cell_spec(self, spec, hxc="scf", fd_nd=4, xc=True, hartree=True) -> int:
        """Register a ``workloads.CellSpec``."""
        return self.add_cell(spec.a, spec.n, spec.atom_frac, spec.n_bands, spec.e_kb_s, spec.e_kb_p,
                             z_ion=spec.z_ion, r_erf=spec.r_erf, c_core=spec.c_core, sigma_core=spec.sigma_core,
                             r_proj=spec.r_proj, proj_half=spec.proj_half, use_projectors=spec.use_projectors,
                             occ=spec.occ, fd_nd=fd_nd, hxc=hxc, xc=xc, hartree=hartree)

    def add_subsim(self, cell_id, kcart, dt, max_steps) -> int:
        k = np.ascontiguousarray(kcart, dtype=np.float64).reshape(-1, 3)
        sid = ctypes.c_int()
        self._check(self.lib.tsbz_add_subsim(self.ctx, cell_id, k.shape[0], _dptr(k), float(dt), int(max_steps),
                                             ctypes.byref(sid)), "tsbz_add_subsim")
        self.subs.append(dict(cell=cell_id, n_k=k.shape[0]))
        return sid.value

    def load_ground_state(self, sid, psi, v_hxc_frozen=None):
        """psi: complex128 numpy array (host) or torch complex128 CUDA tensor (device)."""
        vf = None if v_hxc_frozen is None else np.ascontiguousarray(v_hxc_frozen, dtype=np.float64)
        torch = self._torch
        if isinstance(psi, torch.Tensor):
            assert psi.is_cuda and psi.dtype == torch.complex128 and psi.is_contiguous()
            rc = self.lib.tsbz_load_ground_state(self.ctx, sid, ctypes.c_void_p(psi.data_ptr()), psi.numel(), 1,
                                                 _dptr(vf) if vf is not None else None)
        else:
            p = np.ascontiguousarray(psi, dtype=np.complex128)
            rc = self.lib.tsbz_load_ground_state(self.ctx, sid, p.ctypes.data_as(ctypes.c_void_p), p.size, 0,
                                                 _dptr(vf) if vf is not None else None)
        self._check(rc, "tsbz_load_ground_state")

    def set_kick(self, sid, k0, direction=(1.0, 0.0, 0.0)):
        d = np.ascontiguousarray(direction, dtype=np.float64)
        self._check(self.lib.tsbz_set_kick(self.ctx, sid, float(k0), _dptr(d)), "tsbz_set_kick")

    def set_field(self, sid, samples):
        s = np.ascontiguousarray(samples, dtype=np.float64).reshape(-1, 3)
        n = (s.shape[0] - 1) // 2
        self._check(self.lib.tsbz_set_field(self.ctx, sid, n, _dptr(s)), "tsbz_set_field")

    # -- run -----------------------------------------------------------------
    def propagate(self, n_steps: int):
        self._check(self.lib.tsbz_propagate(self.ctx, int(n_steps)), "tsbz_propagate")

    def current(self, sid, first=0, count=None):
        if count is None:
            count = self.step(sid if sid >= 0 else 0) + 1 - first
        J = np.zeros((count, 3))
        j0 = np.zeros(3)
        self._check(self.lib.tsbz_get_current(self.ctx, sid, first, count, _dptr(J), _dptr(j0)), "tsbz_get_current")
        return J, j0

    def current_stats(self, first=0, count=None):
        """Two-step mean of dJ over the sub-simulations (Eq. 9) and its standard error."""
        if count is None:
            count = min(self.step(i) for i in range(len(self.subs))) + 1 - first
        mean, se = np.zeros((count, 3)), np.zeros((count, 3))
        self._check(self.lib.tsbz_get_current_stats(self.ctx, first, count, _dptr(mean), _dptr(se)),
                    "tsbz_get_current_stats")
        return mean, se

    def density(self, sid):
        c = self.cells[self.subs[sid]["cell"]]
        out = np.zeros(c["n"][::-1])
        self._check(self.lib.tsbz_get_density(self.ctx, sid, _dptr(out), out.size), "tsbz_get_density")
        return out

    def norms(self, sid):
        c = self.cells[self.subs[sid]["cell"]]
        out = np.zeros((self.subs[sid]["n_k"], c["n_bands"]))
        self._check(self.lib.tsbz_get_norms(self.ctx, sid, _dptr(out), out.size), "tsbz_get_norms")
        return out

    def step(self, sid) -> int:
        s = ctypes.c_int()
        self._check(self.lib.tsbz_get_step(self.ctx, sid, ctypes.byref(s)), "tsbz_get_step")
        return s.value

    def get_state(self, sid):
        c = self.cells[self.subs[sid]["cell"]]
        out = np.zeros((self.subs[sid]["n_k"], c["n_bands"]) + c["n"][::-1], dtype=np.complex128)
        st = ctypes.c_int()
        self._check(self.lib.tsbz_get_state(self.ctx, sid, out.ctypes.data_as(_D), out.size, ctypes.byref(st)),
                    "tsbz_get_state")
        return out, st.value

    def load_state(self, sid, psi, step):
        p = np.ascontiguousarray(psi, dtype=np.complex128)
        self._check(self.lib.tsbz_load_state(self.ctx, sid, p.ctypes.data_as(_D), p.size, int(step)),
                    "tsbz_load_state")

    def cell_tables(self, cell_id):
        c = self.cells[cell_id]
        v = np.zeros(c["n"][::-1])
        pn = np.zeros(max(1, 4 * c["n_atoms"]))
        self._check(self.lib.tsbz_get_cell_tables(self.ctx, cell_id, _dptr(v), v.size, _dptr(pn), pn.size),
                    "tsbz_get_cell_tables")
        return v, pn[: 4 * c["n_atoms"]]

    def launches(self) -> int:
        n = ctypes.c_longlong()
        self._check(self.lib.tsbz_get_launch_count(self.ctx, ctypes.byref(n)), "tsbz_get_launch_count")
        return n.value

    def set_graphs(self, on: bool):
        self._check(self.lib.tsbz_set_graphs(self.ctx, 1 if on else 0), "tsbz_set_graphs")

    def set_profiling(self, on: bool):
        self._check(self.lib.tsbz_set_profiling(self.ctx, 1 if on else 0), "tsbz_set_profiling")

    def ground_state(self, max_iter: int = 80, tol: float = 1e-9, degree: int = 48, mix: float = 0.35):
        """Solve the Kohn-Sham ground state of every sub-simulation on the GPU from the
        loaded starting orbitals; returns (iterations, final density error)."""
        it, err = ctypes.c_int(), ctypes.c_double()
        self._check(self.lib.tsbz_ground_state(self.ctx, int(max_iter), float(tol), int(degree), float(mix),
                                               ctypes.byref(it), ctypes.byref(err)), "tsbz_ground_state")
        return it.value, err.value

    def set_propagator(self, name: str):
        """"taylor4" (default) or "etrs"."""
        code = {"taylor4": 0, "etrs": 1}[name]
        self._check(self.lib.tsbz_set_propagator(self.ctx, code), "tsbz_set_propagator")

    def autotune(self, budget_ms: int = 2000) -> int:
        """Time the kernel variants of every cell and keep the fastest (the
        state is restored afterwards); returns the number of variants timed."""
        n = ctypes.c_int()
        self._check(self.lib.tsbz_autotune(self.ctx, int(budget_ms), ctypes.byref(n)), "tsbz_autotune")
        return n.value

    def variant(self, cell_id):
        """(variant in force, number of variants, measured ms per step of each)."""
        v, nv = ctypes.c_int(), ctypes.c_int()
        ms = np.zeros(4)
        self._check(self.lib.tsbz_get_variant(self.ctx, cell_id, ctypes.byref(v), ctypes.byref(nv), _dptr(ms), 4),
                    "tsbz_get_variant")
        return v.value, nv.value, ms[: nv.value].tolist()

    def set_variant(self, cell_id, variant: int):
        self._check(self.lib.tsbz_set_variant(self.ctx, cell_id, int(variant)), "tsbz_set_variant")

    def timings(self):
        t = np.zeros(7)
        self._check(self.lib.tsbz_get_timings(self.ctx, _dptr(t), 7), "tsbz_get_timings")
        return dict(zip(["bra", "stage", "observe", "finalize", "hxc", "field", "ket"], t.tolist()))
