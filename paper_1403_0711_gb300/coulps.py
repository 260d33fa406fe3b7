"""Python binding of the coulps C ABI (include/coulps.h).

Argument marshalling only: every step of the sampler runs in libcoulps.so.
The module-level functions carry the C names; ``Lattice`` and ``Charges`` wrap
the handles.  PyTorch supplies device memory (its caching allocator is
installed as the library's allocator) and streams.

If libcoulps.so cannot be loaded this module raises on first use; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libcoulps.so"

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENONFINITE, EIO, ECORRUPT, EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
F32, F64 = 0, 1

# Every symbol include/coulps.h declares (checked by the CPU test suite).
EXPORTS = (
    "coulps_error_string", "coulps_version", "coulps_set_allocator",
    "coulps_lattice_create", "coulps_lattice_destroy", "coulps_set_stream",
    "coulps_lattice_info", "coulps_set_tile", "coulps_field_get", "coulps_field_set",
    "coulps_sweep", "coulps_sync", "coulps_charges_create", "coulps_charges_destroy",
    "coulps_measure", "coulps_run", "coulps_estimate", "coulps_estimate_post",
    "coulps_estimate_take", "coulps_samples",
    "coulps_reset_stats", "coulps_checkpoint_save", "coulps_checkpoint_load",
    "coulps_charges_update", "coulps_chain_stats", "coulps_pool_stats", "coulps_set_profiling",
    "coulps_kernel_times", "coulps_measure_static",
    "coulps_batch_create", "coulps_batch_destroy", "coulps_batch_set_tiles",
    "coulps_batch_system_tile", "coulps_batch_info", "coulps_batch_charges", "coulps_batch_sweep",
    "coulps_batch_run", "coulps_batch_sync", "coulps_batch_estimate", "coulps_batch_samples",
    "coulps_batch_field_get", "coulps_cv_pack_weights", "coulps_cv_conv3d",
    "coulps_cv_conv3d_wgrad", "coulps_cv_pack_field", "coulps_cv_activate", "coulps_cv_stein_sum",
    "coulps_set_schedule", "coulps_cv_conv3d_tanh", "coulps_cv_conv3d_tanh_rows",
    "coulps_cv_pack_region",
    "coulps_cv_stein_region", "coulps_cv_region_pack", "coulps_cv_record",
    "coulps_cv_chain_stats", "coulps_cv_estimate",
    "coulps_cv_reset", "coulps_cv_charge_term", "coulps_set_fused", "coulps_set_pass_tile",
    "coulps_measure_sets", "coulps_run_sets", "coulps_gcv_create", "coulps_gcv_destroy",
    "coulps_gcv_info", "coulps_gcv_h", "coulps_gcv_eval", "coulps_gcv_run",
    "coulps_batch_field_set", "coulps_batch_stats", "coulps_batch_reset_stats",
    "coulps_batch_gcv_create", "coulps_batch_gcv_destroy", "coulps_batch_gcv_info",
    "coulps_batch_gcv_h", "coulps_batch_gcv_eval", "coulps_batch_gcv_run", "coulps_batch_gcv_reset",
    "coulps_batch_gcv_stats", "coulps_batch_gcv_estimate",
    "coulps_charges_create_off", "coulps_forces", "coulps_charges_near",
    "coulps_heatbath_noise", "coulps_near_pairs", "coulps_offlattice_corners",
    "coulps_set_streams", "coulps_selftest_wait", "coulps_clear_error",
    "coulps_set_pair_tile", "coulps_pair_tile", "coulps_kernel_times_n",
    "coulps_batch_set_fused", "coulps_batch_set_pass_tiles", "coulps_batch_system_pass_tile",
    "coulps_batch_fused", "coulps_batch_set_pair_tiles", "coulps_batch_system_pair_tile",
)
SCHEDULE_ALIGNED, SCHEDULE_PHASED, SCHEDULE_SHIFTED = 0, 1, 2
STAT_STRIDE = 72


class CoulpsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {error_string(status)} ({status})")


_lib = None
_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_keep = []  # ctypes callbacks must outlive the library's use of them


def load(path: str | Path | None = None):
    """Load libcoulps.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        raise RuntimeError(f"libcoulps.so not found at {p}: build it first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    L = ctypes.CDLL(str(p))
    vp, i32, i64, u64, f64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_double)
    P = ctypes.POINTER
    sig = {
        "coulps_error_string": (ctypes.c_char_p, [i32]),
        "coulps_version": (i32, []),
        "coulps_set_allocator": (i32, [_ALLOC_T, _FREE_T, vp]),
        "coulps_lattice_create": (i32, [i32, i32, i32, i32, i32, u64, vp, P(vp)]),
        "coulps_lattice_destroy": (None, [vp]),
        "coulps_set_stream": (i32, [vp, vp]),
        "coulps_lattice_info": (i32, [vp, P(i64)]),
        "coulps_set_tile": (i32, [vp, i32, i32]),
        "coulps_field_get": (i32, [vp, i32, P(f64)]),
        "coulps_field_set": (i32, [vp, i32, P(f64)]),
        "coulps_sweep": (i32, [vp, i32, i32, i32]),
        "coulps_sync": (i32, [vp]),
        "coulps_charges_create": (i32, [vp, i64, P(ctypes.c_int32), P(f64), i64, P(vp)]),
        "coulps_charges_create_off": (i32, [vp, i64, P(f64), P(f64), i64, ctypes.c_int, P(vp)]),
        "coulps_forces": (i32, [vp, P(f64), P(f64)]),
        "coulps_charges_near": (i32, [vp, ctypes.c_double, P(i64), P(f64), P(f64)]),
        "coulps_heatbath_noise": (i32, [i32, vp, vp, i64, vp]),
        "coulps_set_streams": (i32, [vp, i32]),
        "coulps_selftest_wait": (i32, [vp, i64]),
        "coulps_clear_error": (i32, [vp]),
        "coulps_near_pairs": (i32, [i64, P(f64), ctypes.c_double, P(i64), P(ctypes.c_uint32), i64,
                                    P(i64)]),
        "coulps_offlattice_corners": (i32, [i32, i32, i32, i32, i64, P(f64),
                                            P(ctypes.c_uint32), P(f64), P(f64)]),
        "coulps_charges_destroy": (None, [vp]),
        "coulps_measure": (i32, [vp, vp]),
        "coulps_run": (i32, [vp, vp, i32, i32, i32, i32]),
        "coulps_estimate": (i32, [vp, P(f64), P(f64), P(f64), P(i64)]),
        "coulps_estimate_post": (i32, [vp]),
        "coulps_estimate_take": (i32, [vp, P(f64), P(f64), P(f64), P(i64)]),
        "coulps_samples": (i32, [vp, P(f64), i64, P(i64)]),
        "coulps_reset_stats": (i32, [vp]),
        "coulps_checkpoint_save": (i32, [vp, vp, ctypes.c_char_p]),
        "coulps_checkpoint_load": (i32, [vp, vp, ctypes.c_char_p]),
        "coulps_charges_update": (i32, [vp, P(ctypes.c_int32), P(f64)]),
        "coulps_chain_stats": (i32, [vp, P(f64), i64]),
        "coulps_pool_stats": (i32, [P(f64), i64, P(f64), P(f64), P(f64), P(i64)]),
        "coulps_set_profiling": (i32, [vp, i32]),
        "coulps_kernel_times": (i32, [vp, P(f64)]),
        "coulps_measure_static": (i32, [vp, i32, i32, i32, i32, i32, vp, vp, i64, vp, vp]),
        "coulps_batch_create": (i32, [i32, P(ctypes.c_int32), i32, u64, vp, P(vp)]),
        "coulps_batch_destroy": (None, [vp]),
        "coulps_batch_set_tiles": (i32, [vp, P(ctypes.c_int32)]),
        "coulps_batch_system_tile": (i32, [vp, i32, P(ctypes.c_int32)]),
        "coulps_batch_set_fused": (i32, [vp, i32]),
        "coulps_batch_set_pass_tiles": (i32, [vp, P(ctypes.c_int32)]),
        "coulps_batch_system_pass_tile": (i32, [vp, i32, P(ctypes.c_int32)]),
        "coulps_batch_fused": (i32, [vp]),
        "coulps_batch_set_pair_tiles": (i32, [vp, P(ctypes.c_int32)]),
        "coulps_batch_system_pair_tile": (i32, [vp, i32, P(ctypes.c_int32)]),
        "coulps_batch_info": (i32, [vp, P(i64)]),
        "coulps_batch_charges": (i32, [vp, P(i64), P(ctypes.c_int32), P(f64), i64]),
        "coulps_batch_sweep": (i32, [vp, i32, i32, i32]),
        "coulps_batch_run": (i32, [vp, i32, i32, i32, i32]),
        "coulps_batch_sync": (i32, [vp]),
        "coulps_batch_estimate": (i32, [vp, P(f64), P(f64), P(f64), P(i64)]),
        "coulps_batch_samples": (i32, [vp, P(f64), i64, P(i64)]),
        "coulps_batch_field_get": (i32, [vp, i32, P(f64)]),
        "coulps_cv_pack_weights": (i32, [P(ctypes.c_float), P(ctypes.c_uint16)]),
        "coulps_cv_conv3d": (i32, [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]),
        "coulps_cv_conv3d_wgrad": (i32, [vp, vp, vp, i32, i32, i32, i32, vp, i64, vp]),
        "coulps_cv_pack_field": (i32, [vp, vp, vp, vp]),
        "coulps_cv_activate": (i32, [vp, vp, vp, i64, vp]),
        "coulps_cv_stein_sum": (i32, [vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, vp, i64, vp, vp]),
        "coulps_set_schedule": (i32, [vp, i32]),
        "coulps_cv_conv3d_tanh": (i32, [vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]),
        "coulps_cv_conv3d_tanh_rows": (i32, [vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32,
                                             i32, i32, vp, vp]),
        "coulps_cv_pack_region": (i32, [vp, vp, P(ctypes.c_int32), P(ctypes.c_int32), i32, vp,
                                        vp]),
        "coulps_cv_region_pack": (i32, [vp, vp, vp]),
        "coulps_cv_stein_region": (i32, [vp, vp, ctypes.c_float, vp, vp, vp, vp, i32,
                                         P(ctypes.c_int32), i32, P(ctypes.c_int32),
                                         P(ctypes.c_int32), vp, i64, vp, vp, vp]),
        "coulps_cv_record": (i32, [vp, vp, f64]),
        "coulps_cv_chain_stats": (i32, [vp, P(f64), i64]),
        "coulps_cv_estimate": (i32, [vp, P(f64), P(f64), P(f64), P(i64)]),
        "coulps_cv_reset": (i32, [vp]),
        "coulps_set_fused": (i32, [vp, i32]),
        "coulps_measure_sets": (i32, [vp, P(vp), i32]),
        "coulps_gcv_create": (i32, [vp, i32, i32, P(vp)]),
        "coulps_gcv_destroy": (None, [vp]),
        "coulps_gcv_info": (i32, [vp, P(f64)]),
        "coulps_gcv_h": (i32, [vp, P(ctypes.c_float)]),
        "coulps_gcv_eval": (i32, [vp, vp]),
        "coulps_gcv_run": (i32, [vp, i32, i32, i32, f64]),
        "coulps_batch_field_set": (i32, [vp, i32, P(f64)]),
        "coulps_batch_stats": (i32, [vp, P(f64), i64]),
        "coulps_batch_reset_stats": (i32, [vp]),
        "coulps_batch_gcv_create": (i32, [vp, i32, i32, P(vp)]),
        "coulps_batch_gcv_destroy": (None, [vp]),
        "coulps_batch_gcv_info": (i32, [vp, P(f64)]),
        "coulps_batch_gcv_h": (i32, [vp, i32, P(ctypes.c_float)]),
        "coulps_batch_gcv_eval": (i32, [vp, vp]),
        "coulps_batch_gcv_run": (i32, [vp, i32, i32, i32, f64]),
        "coulps_batch_gcv_reset": (i32, [vp]),
        "coulps_batch_gcv_stats": (i32, [vp, P(f64), i64]),
        "coulps_batch_gcv_estimate": (i32, [vp, P(f64), P(f64), P(f64), P(i64)]),
        "coulps_run_sets": (i32, [vp, P(vp), i32, i32, i32, i32, i32]),
        "coulps_set_pass_tile": (i32, [vp, i32, i32]),
        "coulps_set_pair_tile": (i32, [vp, i32, i32]),
        "coulps_pair_tile": (i32, [vp, P(i32)]),
        "coulps_kernel_times_n": (i32, [vp, P(f64), i32]),
        "coulps_cv_charge_term": (i32, [vp, vp, vp, vp, vp, i32, i32, P(ctypes.c_int32), i32, vp,
                                        i64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def error_string(status: int) -> str:
    return load().coulps_error_string(int(status)).decode()


def _check(status: int, where: str):
    if status != OK:
        raise CoulpsError(status, where)


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory: the library reports COULPS_ENOMEM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = _ALLOC_T(_alloc), _FREE_T(_free)
    _keep.extend([a, f])
    _check(load().coulps_set_allocator(a, f, None), "coulps_set_allocator")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# --------------------------------------------------------------------------
class Lattice:
    """n_chains independent chains of phi on an Lx x Ly x Lz Dirichlet box."""

    def __init__(self, L, n_chains=1, precision=F32, seed=0, stream=None):
        self._lib = load()
        self.L = tuple(int(v) for v in L)
        self.n_chains = int(n_chains)
        self.precision = int(precision)
        self.seed = int(seed)
        self._stream = stream
        h = ctypes.c_void_p()
        _check(self._lib.coulps_lattice_create(*self.L, self.n_chains, self.precision,
                                               self.seed, _stream_handle(stream), ctypes.byref(h)),
               "coulps_lattice_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._lib.coulps_lattice_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = (ctypes.c_int64 * 13)()
        _check(self._lib.coulps_lattice_info(self.handle, a), "coulps_lattice_info")
        keys = ("Lx", "Ly", "Lz", "n_chains", "precision", "W", "pass", "bytes", "ty", "dz",
                "fused", "pass_ty", "pass_dz")
        return dict(zip(keys, list(a)))

    def set_stream(self, stream):
        self._stream = stream
        _check(self._lib.coulps_set_stream(self.handle, _stream_handle(stream)), "coulps_set_stream")

    def set_tile(self, ty=0, dz=0):
        _check(self._lib.coulps_set_tile(self.handle, int(ty), int(dz)), "coulps_set_tile")

    def field(self, chain=0):
        Lx, Ly, Lz = self.L
        out = np.empty((Lz, Ly, Lx), dtype=np.float64)
        _check(self._lib.coulps_field_get(self.handle, int(chain), _f64p(out)), "coulps_field_get")
        return out

    def set_field(self, chain, phi):
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        Lx, Ly, Lz = self.L
        assert phi.shape == (Lz, Ly, Lx)
        _check(self._lib.coulps_field_set(self.handle, int(chain), _f64p(phi)), "coulps_field_set")

    def sweep(self, n_compound=1, n_hb=1, n_or=0):
        _check(self._lib.coulps_sweep(self.handle, int(n_compound), int(n_hb), int(n_or)),
               "coulps_sweep")

    def sync(self):
        _check(self._lib.coulps_sync(self.handle), "coulps_sync")

    def selftest_wait(self, limit_ns):
        """Queue a bounded wait that times out (coulps_selftest_wait)."""
        _check(self._lib.coulps_selftest_wait(self.handle, int(limit_ns)), "coulps_selftest_wait")

    def clear_error(self):
        _check(self._lib.coulps_clear_error(self.handle), "coulps_clear_error")

    def set_profiling(self, enable=True):
        _check(self._lib.coulps_set_profiling(self.handle, int(bool(enable))), "coulps_set_profiling")

    def kernel_times(self):
        """{'hb_ms', 'hb_n', 'or_ms', 'or_n', 'mixed_ms', 'mixed_n', 'pass_hb_ms',
        'pass_hb_n', 'pass_or_ms', 'pass_or_n', 'pair_hb_ms', 'pair_hb_n', 'pair_or_ms',
        'pair_or_n'} since the last call (coulps_kernel_times_n)."""
        a = (ctypes.c_double * 14)()
        _check(self._lib.coulps_kernel_times_n(self.handle, a, 14), "coulps_kernel_times_n")
        return {"hb_ms": a[0], "hb_n": int(a[1]), "or_ms": a[2], "or_n": int(a[3]),
                "mixed_ms": a[4], "mixed_n": int(a[5]), "pass_hb_ms": a[6], "pass_hb_n": int(a[7]),
                "pass_or_ms": a[8], "pass_or_n": int(a[9]), "pair_hb_ms": a[10],
                "pair_hb_n": int(a[11]), "pair_or_ms": a[12], "pair_or_n": int(a[13])}

    def set_streams(self, n):
        """1 or 2 streams per compound sweep (coulps_set_streams)."""
        _check(self._lib.coulps_set_streams(self.handle, int(n)), "coulps_set_streams")

    def set_schedule(self, schedule):
        _check(self._lib.coulps_set_schedule(self.handle, int(schedule)), "coulps_set_schedule")

    def set_fused(self, mode):
        """Fused passes (two copies of the field): 0/False off, 1/True the
        over-relaxation passes one kernel per pass, 2 all passes one kernel per
        pass, 3 over-relaxation passes two per kernel (pass pairs), 4 all
        passes as pass pairs (coulps_set_fused)."""
        _check(self._lib.coulps_set_fused(self.handle, int(mode)), "coulps_set_fused")

    def set_pass_tile(self, ty, dz=0):
        _check(self._lib.coulps_set_pass_tile(self.handle, int(ty), int(dz)),
               "coulps_set_pass_tile")

    def set_pair_tile(self, ty, dz=0):
        _check(self._lib.coulps_set_pair_tile(self.handle, int(ty), int(dz)),
               "coulps_set_pair_tile")

    def pair_tile(self):
        a = (ctypes.c_int32 * 2)()
        _check(self._lib.coulps_pair_tile(self.handle, a), "coulps_pair_tile")
        return int(a[0]), int(a[1])

    def checkpoint_save(self, path, charges=None):
        _check(self._lib.coulps_checkpoint_save(self.handle, charges.handle if charges else None,
                                                str(path).encode()), "coulps_checkpoint_save")

    def checkpoint_load(self, path, charges=None):
        _check(self._lib.coulps_checkpoint_load(self.handle, charges.handle if charges else None,
                                                str(path).encode()), "coulps_checkpoint_load")


class Charges:
    """A charge set measured on every chain of a lattice."""

    def __init__(self, lattice: Lattice, sites, q, log_capacity=0, _handle=None):
        self._lib = load()
        self.lattice = lattice
        self.log_capacity = int(log_capacity)
        if _handle is not None:
            self.n = len(q)
            self.handle = _handle
            return
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32).reshape(-1, 3))
        qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
        assert len(s) == len(qq)
        self.n = len(qq)
        h = ctypes.c_void_p()
        _check(self._lib.coulps_charges_create(
            lattice.handle, self.n, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _f64p(qq),
            int(log_capacity), ctypes.byref(h)), "coulps_charges_create")
        self.handle = h

    @classmethod
    def off_lattice(cls, lattice: Lattice, pos, q, log_capacity=0, forces=False):
        """Particles at real positions pos (n, 3) as (x, y, z), each read
        through the trilinear weights of its eight surrounding sites
        (coulps_charges_create_off); forces=True keeps the force sums."""
        lib = load()
        p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
        qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
        assert len(p) == len(qq)
        h = ctypes.c_void_p()
        _check(lib.coulps_charges_create_off(lattice.handle, len(qq), _f64p(p), _f64p(qq),
                                             int(log_capacity), int(bool(forces)),
                                             ctypes.byref(h)), "coulps_charges_create_off")
        return cls(lattice, None, qq, log_capacity=log_capacity, _handle=h)

    def near(self, rc):
        """Leave the pairs closer than rc out of every sample; returns their
        direct (continuum Eq. (s1)) energy and forces to add back."""
        npairs = ctypes.c_int64()
        e = ctypes.c_double()
        f = np.zeros((self.n, 3), dtype=np.float64)
        _check(self._lib.coulps_charges_near(self.handle, float(rc), ctypes.byref(npairs),
                                             ctypes.byref(e), _f64p(f)), "coulps_charges_near")
        return {"n_pairs": npairs.value, "e_direct": e.value, "f_direct": f}

    def forces(self):
        """(mean (n, 3), stderr over chains (n, 3)) of -de/dr_i."""
        m = np.empty((self.n, 3), dtype=np.float64)
        e = np.empty((self.n, 3), dtype=np.float64)
        _check(self._lib.coulps_forces(self.handle, _f64p(m), _f64p(e)), "coulps_forces")
        return m, e

    def close(self):
        if getattr(self, "handle", None):
            self._lib.coulps_charges_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def measure(self):
        _check(self._lib.coulps_measure(self.lattice.handle, self.handle), "coulps_measure")

    def run(self, n_therm, n_meas, n_hb=1, n_or=0):
        _check(self._lib.coulps_run(self.lattice.handle, self.handle, int(n_therm), int(n_meas),
                                    int(n_hb), int(n_or)), "coulps_run")

    def estimate(self):
        m, s, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(self._lib.coulps_estimate(self.handle, ctypes.byref(m), ctypes.byref(s),
                                         ctypes.byref(t), ctypes.byref(n)), "coulps_estimate")
        return {"mean": m.value, "stderr": s.value, "tau_int": t.value, "n": n.value}

    def estimate_post(self):
        """Queue a copy of the estimator state as of everything queued so far
        (coulps_estimate_post); at most two outstanding."""
        _check(self._lib.coulps_estimate_post(self.handle), "coulps_estimate_post")

    def estimate_take(self):
        """The estimate of the oldest posted state (coulps_estimate_take)."""
        m, s, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(self._lib.coulps_estimate_take(self.handle, ctypes.byref(m), ctypes.byref(s),
                                              ctypes.byref(t), ctypes.byref(n)),
               "coulps_estimate_take")
        return {"mean": m.value, "stderr": s.value, "tau_int": t.value, "n": n.value}

    def samples(self, cap=None):
        """(n_samples, n_chains, 3) array of logged (Q, P, e)."""
        nc = self.lattice.n_chains
        if cap is None:
            cap = max(1, self.log_capacity)
        buf = np.empty((cap, nc, 3), dtype=np.float64)
        n = ctypes.c_int64()
        _check(self._lib.coulps_samples(self.handle, _f64p(buf), int(cap), ctypes.byref(n)),
               "coulps_samples")
        return buf[: n.value].copy()

    def reset_stats(self):
        _check(self._lib.coulps_reset_stats(self.handle), "coulps_reset_stats")

    def update(self, sites, q):
        """Replace the charges' positions and values (same count)."""
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32).reshape(-1, 3))
        qq = np.ascontiguousarray(np.asarray(q, dtype=np.float64).reshape(-1))
        assert len(s) == len(qq) == self.n
        _check(self._lib.coulps_charges_update(
            self.handle, s.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _f64p(qq)),
            "coulps_charges_update")

    def chain_stats(self):
        """(n_chains, STAT_STRIDE) raw per-chain estimator state."""
        nc = self.lattice.n_chains
        out = np.empty((nc, STAT_STRIDE), dtype=np.float64)
        _check(self._lib.coulps_chain_stats(self.handle, _f64p(out), out.size), "coulps_chain_stats")
        return out

    # control-variate samples y = e - c * Tg, kept beside the plain ones
    def cv_record(self, tg_ptr, c):
        """Record y_b = e_b - c * tg[b] for every chain (tg: device doubles)."""
        _check(self._lib.coulps_cv_record(self.handle, ctypes.c_void_p(tg_ptr), float(c)),
               "coulps_cv_record")

    def cv_estimate(self):
        m, s, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int64()
        _check(self._lib.coulps_cv_estimate(self.handle, ctypes.byref(m), ctypes.byref(s),
                                            ctypes.byref(t), ctypes.byref(n)), "coulps_cv_estimate")
        return {"mean": m.value, "stderr": s.value, "tau_int": t.value, "n": n.value}

    def cv_chain_stats(self):
        nc = self.lattice.n_chains
        out = np.empty((nc, STAT_STRIDE), dtype=np.float64)
        _check(self._lib.coulps_cv_chain_stats(self.handle, _f64p(out), out.size),
               "coulps_cv_chain_stats")
        return out

    def cv_reset(self):
        _check(self._lib.coulps_cv_reset(self.handle), "coulps_cv_reset")


class GlobalCV:
    """Global control variate g = Q h of a charge set (coulps_gcv_*): h from
    n_iter SOR iterations on A h = -rho; with R > 0 also the local term of P
    (kernel radius R)."""

    def __init__(self, charges, n_iter=None, R=1):
        self.charges = charges
        self._lib = load()
        L = charges.lattice.L
        if n_iter is None:
            n_iter = 6 * max(L) + 50
        h = ctypes.c_void_p()
        _check(self._lib.coulps_gcv_create(charges.handle, int(n_iter), int(R), ctypes.byref(h)),
               "coulps_gcv_create")
        self.handle = h

    def close(self):
        if self.handle:
            self._lib.coulps_gcv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = (ctypes.c_double * 2)()
        _check(self._lib.coulps_gcv_info(self.handle, a), "coulps_gcv_info")
        return {"h_dot_rho": a[0], "residual": a[1]}

    def h(self):
        Lx, Ly, Lz = self.charges.lattice.L
        out = np.empty((Lz, Ly, Lx), dtype=np.float32)
        _check(self._lib.coulps_gcv_h(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "coulps_gcv_h")
        return out

    def eval(self, tg_ptr=None):
        """T g of the current fields into device doubles at tg_ptr (None: internal)."""
        _check(self._lib.coulps_gcv_eval(self.handle, ctypes.c_void_p(tg_ptr) if tg_ptr else None),
               "coulps_gcv_eval")

    def run(self, n_meas, n_hb=1, n_or=0, c=1.0):
        _check(self._lib.coulps_gcv_run(self.handle, int(n_meas), int(n_hb), int(n_or), float(c)),
               "coulps_gcv_run")


def _set_array(sets):
    arr = (ctypes.c_void_p * len(sets))(*[c.handle for c in sets])
    return arr


def measure_sets(lattice, sets):
    """One sample of every charge set (all of `lattice`) from the current fields."""
    sets = list(sets)
    _check(load().coulps_measure_sets(lattice.handle, _set_array(sets), len(sets)),
           "coulps_measure_sets")


def run_sets(lattice, sets, n_therm, n_meas, n_hb=1, n_or=0):
    """n_therm + n_meas compound sweeps; every measured one samples every set."""
    sets = list(sets)
    _check(load().coulps_run_sets(lattice.handle, _set_array(sets), len(sets), int(n_therm),
                                  int(n_meas), int(n_hb), int(n_or)), "coulps_run_sets")


def pool_stats(rows):
    """Pool per-chain estimator rows (any number, e.g. gathered from several
    processes) exactly as Charges.estimate does."""
    rows = np.ascontiguousarray(np.asarray(rows, dtype=np.float64).reshape(-1, STAT_STRIDE))
    m, s, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().coulps_pool_stats(_f64p(rows), len(rows), ctypes.byref(m), ctypes.byref(s),
                                    ctypes.byref(t), ctypes.byref(n)), "coulps_pool_stats")
    return {"mean": m.value, "stderr": s.value, "tau_int": t.value, "n": n.value}


class Batch:
    """Many independent one-chain systems of different shapes, swept together."""

    def __init__(self, dims, precision=F32, seed=0, stream=None):
        self._lib = load()
        d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32).reshape(-1, 3))
        self.dims = [tuple(int(v) for v in r) for r in d]
        self.n = len(d)
        self.precision = int(precision)
        h = ctypes.c_void_p()
        _check(self._lib.coulps_batch_create(self.n, d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                             self.precision, int(seed), _stream_handle(stream),
                                             ctypes.byref(h)), "coulps_batch_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            self._lib.coulps_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = (ctypes.c_int64 * 10)()
        _check(self._lib.coulps_batch_info(self.handle, a), "coulps_batch_info")
        keys = ("n_systems", "tiles", "grid", "smem", "pass", "field_bytes", "sites",
                "pass_grid", "pair_grid", "pair_threads")
        return dict(zip(keys, list(a)))

    def set_tiles(self, ty_dz):
        t = np.ascontiguousarray(np.asarray(ty_dz, dtype=np.int32).reshape(-1, 2))
        assert len(t) == self.n
        _check(self._lib.coulps_batch_set_tiles(self.handle, t.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int32))), "coulps_batch_set_tiles")

    def tiles(self):
        out = []
        for s in range(self.n):
            a = (ctypes.c_int32 * 2)()
            _check(self._lib.coulps_batch_system_tile(self.handle, s, a), "coulps_batch_system_tile")
            out.append((a[0], a[1]))
        return out

    def set_fused(self, mode):
        """Over-relaxation passes as half-sweeps only (0), fused passes (1) or
        pass pairs (2, the default where every system admits a pair tile); 3:
        all passes, heatbath ones included, as pass pairs and fused passes."""
        _check(self._lib.coulps_batch_set_fused(self.handle, int(mode)), "coulps_batch_set_fused")

    def fused(self):
        return int(self._lib.coulps_batch_fused(self.handle))

    def set_pair_tiles(self, ty_dz):
        t = np.ascontiguousarray(np.asarray(ty_dz, dtype=np.int32).reshape(-1, 2))
        assert len(t) == self.n
        _check(self._lib.coulps_batch_set_pair_tiles(self.handle, t.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int32))), "coulps_batch_set_pair_tiles")

    def pair_tiles(self):
        out = []
        for s in range(self.n):
            a = (ctypes.c_int32 * 2)()
            _check(self._lib.coulps_batch_system_pair_tile(self.handle, s, a),
                   "coulps_batch_system_pair_tile")
            out.append((a[0], a[1]))
        return out

    def set_pass_tiles(self, ty_dz):
        t = np.ascontiguousarray(np.asarray(ty_dz, dtype=np.int32).reshape(-1, 2))
        assert len(t) == self.n
        _check(self._lib.coulps_batch_set_pass_tiles(self.handle, t.ctypes.data_as(
            ctypes.POINTER(ctypes.c_int32))), "coulps_batch_set_pass_tiles")

    def pass_tiles(self):
        out = []
        for s in range(self.n):
            a = (ctypes.c_int32 * 2)()
            _check(self._lib.coulps_batch_system_pass_tile(self.handle, s, a),
                   "coulps_batch_system_pass_tile")
            out.append((a[0], a[1]))
        return out

    def set_charges(self, systems, log_capacity=0):
        """systems: list of (sites, q), one per system."""
        assert len(systems) == self.n
        offs = np.zeros(self.n + 1, dtype=np.int64)
        for i, (s_, q_) in enumerate(systems):
            offs[i + 1] = offs[i] + len(q_)
        sites = np.ascontiguousarray(np.concatenate(
            [np.asarray(s_, dtype=np.int32).reshape(-1, 3) for s_, _ in systems]))
        q = np.ascontiguousarray(np.concatenate(
            [np.asarray(q_, dtype=np.float64).reshape(-1) for _, q_ in systems]))
        self.log_capacity = int(log_capacity)
        _check(self._lib.coulps_batch_charges(
            self.handle, offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            sites.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _f64p(q), int(log_capacity)),
            "coulps_batch_charges")

    def sweep(self, n_compound=1, n_hb=1, n_or=0):
        _check(self._lib.coulps_batch_sweep(self.handle, int(n_compound), int(n_hb), int(n_or)),
               "coulps_batch_sweep")

    def run(self, n_therm, n_meas, n_hb=1, n_or=0):
        _check(self._lib.coulps_batch_run(self.handle, int(n_therm), int(n_meas), int(n_hb),
                                          int(n_or)), "coulps_batch_run")

    def sync(self):
        _check(self._lib.coulps_batch_sync(self.handle), "coulps_batch_sync")

    def estimate(self):
        m, s, t = (np.empty(self.n) for _ in range(3))
        n = np.empty(self.n, dtype=np.int64)
        _check(self._lib.coulps_batch_estimate(self.handle, _f64p(m), _f64p(s), _f64p(t),
                                               n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "coulps_batch_estimate")
        return {"mean": m, "stderr": s, "tau_int": t, "n": n}

    def samples(self, cap=None):
        """(n_samples, n_systems, 3) array of logged (Q, P, e)."""
        cap = self.log_capacity if cap is None else cap
        buf = np.empty((max(1, cap), self.n, 3))
        n = ctypes.c_int64()
        _check(self._lib.coulps_batch_samples(self.handle, _f64p(buf), int(cap), ctypes.byref(n)),
               "coulps_batch_samples")
        return buf[: n.value].copy()

    def field(self, system):
        Lx, Ly, Lz = self.dims[system]
        out = np.empty((Lz, Ly, Lx))
        _check(self._lib.coulps_batch_field_get(self.handle, int(system), _f64p(out)),
               "coulps_batch_field_get")
        return out

    def set_field(self, system, phi):
        """phi: (Lz, Ly, Lx) array, x fastest."""
        Lx, Ly, Lz = self.dims[system]
        a = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(Lz, Ly, Lx))
        _check(self._lib.coulps_batch_field_set(self.handle, int(system), _f64p(a)),
               "coulps_batch_field_set")

    def stats(self):
        """(n_systems, COULPS_STAT_STRIDE) raw statistics of the plain samples."""
        out = np.empty((self.n, STAT_STRIDE))
        _check(self._lib.coulps_batch_stats(self.handle, _f64p(out), out.size), "coulps_batch_stats")
        return out

    def reset_stats(self):
        _check(self._lib.coulps_batch_reset_stats(self.handle), "coulps_batch_reset_stats")


class BatchGlobalCV:
    """Global control variate of every system of a Batch (coulps_batch_gcv_*):
    per system h from n_iter SOR iterations on A h = -rho; with R > 0 also
    the local term of P (kernel radius R)."""

    def __init__(self, batch, n_iter=None, R=1):
        self.batch = batch
        self._lib = load()
        if n_iter is None:
            n_iter = 6 * max(max(L) for L in batch.dims) + 50
        h = ctypes.c_void_p()
        _check(self._lib.coulps_batch_gcv_create(batch.handle, int(n_iter), int(R), ctypes.byref(h)),
               "coulps_batch_gcv_create")
        self.handle = h

    def close(self):
        if self.handle:
            self._lib.coulps_batch_gcv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = np.empty(2 * self.batch.n)
        _check(self._lib.coulps_batch_gcv_info(self.handle, _f64p(a)), "coulps_batch_gcv_info")
        return {"h_dot_rho": a[0::2].copy(), "residual": a[1::2].copy()}

    def h(self, system):
        Lx, Ly, Lz = self.batch.dims[system]
        out = np.empty((Lz, Ly, Lx), dtype=np.float32)
        _check(self._lib.coulps_batch_gcv_h(self.handle, int(system),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "coulps_batch_gcv_h")
        return out

    def eval(self, tg_ptr=None):
        """T g of every system's field into device doubles at tg_ptr (None: internal)."""
        _check(self._lib.coulps_batch_gcv_eval(self.handle,
                                               ctypes.c_void_p(tg_ptr) if tg_ptr else None),
               "coulps_batch_gcv_eval")

    def run(self, n_meas, n_hb=1, n_or=3, c=1.0):
        _check(self._lib.coulps_batch_gcv_run(self.handle, int(n_meas), int(n_hb), int(n_or),
                                              float(c)), "coulps_batch_gcv_run")

    def reset(self):
        _check(self._lib.coulps_batch_gcv_reset(self.handle), "coulps_batch_gcv_reset")

    def stats(self):
        out = np.empty((self.batch.n, STAT_STRIDE))
        _check(self._lib.coulps_batch_gcv_stats(self.handle, _f64p(out), out.size),
               "coulps_batch_gcv_stats")
        return out

    def estimate(self):
        m, s, t = (np.empty(self.batch.n) for _ in range(3))
        n = np.empty(self.batch.n, dtype=np.int64)
        _check(self._lib.coulps_batch_gcv_estimate(self.handle, _f64p(m), _f64p(s), _f64p(t),
                                                   n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))),
               "coulps_batch_gcv_estimate")
        return {"mean": m, "stderr": s, "tau_int": t, "n": n}


# C-named module functions -------------------------------------------------
def coulps_lattice_create(Lx, Ly, Lz, n_chains, precision, seed, stream=None):
    return Lattice((Lx, Ly, Lz), n_chains, precision, seed, stream)


def coulps_charges_create(lattice, sites, q, log_capacity=0):
    return Charges(lattice, sites, q, log_capacity)


def coulps_charges_create_off(lattice, pos, q, log_capacity=0, forces=False):
    return Charges.off_lattice(lattice, pos, q, log_capacity, forces)


def coulps_forces(charges):
    return charges.forces()


def coulps_charges_near(charges, rc):
    return charges.near(rc)


def near_pairs(pos, rc):
    """CSR (ptr, nbr) of the near partners of particles at pos (n, 3)
    (coulps_near_pairs; host only)."""
    lib = load()
    p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    n = len(p)
    ptr = np.zeros(n + 1, dtype=np.int64)
    need = ctypes.c_int64()
    st = lib.coulps_near_pairs(n, _f64p(p), float(rc), ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               None, 0, ctypes.byref(need))
    if st == 0:
        return ptr, np.zeros(0, dtype=np.uint32)
    nbr = np.zeros(need.value, dtype=np.uint32)
    _check(lib.coulps_near_pairs(n, _f64p(p), float(rc),
                                 ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                 nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), len(nbr),
                                 ctypes.byref(need)), "coulps_near_pairs")
    return ptr, nbr


def offlattice_corners(L, precision, pos):
    """(offset (n, 8), weight (n, 8), grad (n, 8, 3)) of coulps_offlattice_corners."""
    lib = load()
    p = np.ascontiguousarray(np.asarray(pos, dtype=np.float64).reshape(-1, 3))
    n = len(p)
    off = np.zeros((n, 8), dtype=np.uint32)
    w = np.zeros((n, 8))
    g = np.zeros((n, 8, 3))
    _check(lib.coulps_offlattice_corners(int(L[0]), int(L[1]), int(L[2]), int(precision), n,
                                         _f64p(p), off.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                         _f64p(w), _f64p(g)), "coulps_offlattice_corners")
    return off, w, g


def heatbath_noise(words, precision, stream=None):
    """The heatbath's random term for 32-bit words (coulps_heatbath_noise):
    words is a CUDA tensor of int32 (the words' bit patterns); returns a
    float32 / float64 CUDA tensor."""
    import torch
    lib = load()
    w = words.contiguous()
    dt = torch.float32 if precision == F32 else torch.float64
    out = torch.empty(w.shape, dtype=dt, device=w.device)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream(w.device).cuda_stream
    _check(lib.coulps_heatbath_noise(int(precision), ctypes.c_void_p(w.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), w.numel(), ctypes.c_void_p(s)),
           "coulps_heatbath_noise")
    return out


def coulps_sweep(lattice, n_compound, n_hb, n_or):
    lattice.sweep(n_compound, n_hb, n_or)


def coulps_measure(lattice, charges):
    assert charges.lattice is lattice
    charges.measure()


def coulps_run(lattice, charges, n_therm, n_meas, n_hb, n_or):
    assert charges.lattice is lattice
    charges.run(n_therm, n_meas, n_hb, n_or)


def coulps_estimate(charges):
    return charges.estimate()


def coulps_samples(charges, cap=None):
    return charges.samples(cap)


def coulps_field_get(lattice, chain):
    return lattice.field(chain)


def coulps_field_set(lattice, chain, phi):
    lattice.set_field(chain, phi)
