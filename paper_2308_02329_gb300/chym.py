"""Thin ctypes binding of the C ABI in ``include/chym.h``.

Argument marshalling only: every step of the simulation runs in the CUDA
library.  The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2308_02329_gb300.build``); a missing library raises, there is
no fallback.  Device pointers and CUDA streams may come from torch
(``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``) or any
other CUDA runtime user.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libchym.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTSUP, ESTATE = range(7)
J_PM1, J_REAL = 0, 1
PREC_FP64, PREC_FP32, PREC_BF16X2, PREC_FP8 = 0, 1, 2, 3
FLAG_TEST_STALL = 1
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENOTSUP", 6: "ESTATE"}

EXPORTS = ["chym_last_error", "chym_create", "chym_destroy", "chym_lambda_max", "chym_run",
           "chym_run_device", "chym_energy", "chym_energy_device", "chym_readout_xy",
           "chym_readout_xy_device", "chym_stats", "chym_set_coupling_weights",
           "chym_energy_segments",
           "chym_get_state", "chym_set_state", "chym_info", "chym_ground_state_exact",
           "chym_ground_state_mobius", "chym_ground_state_search", "chym_stats_noalloc",
           "chym_batch_create", "chym_batch_run", "chym_batch_status", "chym_batch_destroy",
           "chym_batch_tune", "chym_batch_get_tuning", "chym_batch_set_tuning",
           "chym_batch_get_shapes", "chym_batch_set_shapes", "chym_checkpoint", "chym_restore",
           "chym_exit_scan_device",
           "chym_reseed_device", "chym_get_offsets_device", "chym_copy_state_device",
           "chym_features_device", "chym_mlp_create", "chym_mlp_destroy", "chym_mlp_set_params",
           "chym_mlp_get_params", "chym_mlp_forward_device", "chym_mlp_grad_device",
           "chym_mlp_train_step_device"]


class ChymError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class CParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("sigma", ctypes.c_double),
                ("init_std", ctypes.c_double), ("gamma", ctypes.c_double),
                ("kappa", ctypes.c_double), ("eps", ctypes.c_double),
                ("prec", ctypes.c_int32), ("flags", ctypes.c_int32)]


class CSchedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("k_anneal", ctypes.c_int64), ("k_total", ctypes.c_int64)]


class CStats(ctypes.Structure):
    _fields_ = [("P_max", ctypes.c_double), ("W_range", ctypes.c_double),
                ("W_scan", ctypes.c_double), ("dE_mean", ctypes.c_double),
                ("best_E", ctypes.c_double), ("best_run", ctypes.c_int64),
                ("n_finite", ctypes.c_int64), ("n_hits", ctypes.c_int64)]


@dataclass
class Params:
    """Model constants (see include/chym.h): gamma = beta b^2, kappa = kappa L."""
    dt: float = 0.01
    sigma: float = 1e-3
    init_std: float = 0.1
    gamma: float = 25.0
    kappa: float = 0.1
    eps: float = 0.05
    prec: int = PREC_FP32
    flags: int = 0   # FLAG_TEST_STALL only in tests of the timeout path

    def c(self):
        return CParams(self.dt, self.sigma, self.init_std, self.gamma, self.kappa, self.eps,
                       int(self.prec), int(self.flags))


@dataclass
class Schedule:
    kind: int = 1
    k_anneal: int = 0
    k_total: int = 1

    def c(self):
        return CSchedule(int(self.kind), 0, int(self.k_anneal), int(self.k_total))


_lib = None


def lib():
    """Load libchym.so once; raise if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"CHYM CUDA library not built: {LIB_PATH} is missing "
                              "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        L.chym_last_error.restype = ctypes.c_char_p
        L.chym_last_error.argtypes = []
        L.chym_create.argtypes = [vp, i32, i32, i32, ctypes.POINTER(vp)]
        L.chym_destroy.argtypes = [vp]
        L.chym_lambda_max.argtypes = [vp, ctypes.POINTER(dbl)]
        L.chym_run.argtypes = [vp, ctypes.POINTER(CParams), vp, i32, vp, i32, i64,
                               ctypes.POINTER(CSchedule), vp]
        L.chym_run_device.argtypes = L.chym_run.argtypes
        L.chym_energy.argtypes = [vp, vp, vp, vp]
        L.chym_energy_device.argtypes = [vp, vp, vp, vp]
        L.chym_readout_xy.argtypes = [vp, vp, vp, vp]
        L.chym_set_coupling_weights.argtypes = [vp, vp]
        L.chym_energy_segments.argtypes = [vp, i32, vp, vp, vp]
        L.chym_readout_xy_device.argtypes = [vp, vp, vp, vp]
        L.chym_stats.argtypes = [vp, dbl, ctypes.POINTER(CStats), vp, vp, i32, vp]
        L.chym_get_state.argtypes = [vp, vp, ctypes.POINTER(i64), vp]
        L.chym_set_state.argtypes = [vp, vp, i32, vp, i32, vp, i64, ctypes.c_int32, vp]
        L.chym_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]
        L.chym_ground_state_exact.argtypes = [vp, ctypes.POINTER(dbl), vp]
        L.chym_ground_state_mobius.argtypes = [i32, dbl, dbl, ctypes.POINTER(dbl)]
        L.chym_ground_state_search.argtypes = [vp, i32, i32, ctypes.c_uint64, ctypes.POINTER(dbl), vp]
        L.chym_reseed_device.argtypes = [vp, vp, i32, vp, vp, dbl, vp]
        L.chym_get_offsets_device.argtypes = [vp, vp, vp]
        L.chym_copy_state_device.argtypes = [vp, vp, vp]
        L.chym_features_device.argtypes = [vp, vp, dbl, vp, vp]
        L.chym_mlp_create.argtypes = [ctypes.c_uint64, i32, ctypes.POINTER(vp)]
        L.chym_mlp_destroy.argtypes = [vp]
        L.chym_mlp_set_params.argtypes = [vp, vp, vp, vp]
        L.chym_mlp_get_params.argtypes = [vp, vp]
        L.chym_mlp_forward_device.argtypes = [vp, vp, i32, vp, vp]
        L.chym_mlp_grad_device.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.chym_mlp_train_step_device.argtypes = [vp, vp, vp, i32, ctypes.c_float, vp, vp]
        L.chym_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
        L.chym_batch_run.argtypes = [vp, ctypes.POINTER(CParams), ctypes.POINTER(CSchedule), i64, vp]
        L.chym_batch_status.argtypes = [vp]
        L.chym_batch_destroy.argtypes = [vp]
        L.chym_batch_tune.argtypes = [vp, ctypes.POINTER(CParams), ctypes.POINTER(CSchedule), i64, vp]
        L.chym_batch_get_tuning.argtypes = [vp, vp, ctypes.POINTER(dbl), ctypes.POINTER(i32)]
        L.chym_batch_set_tuning.argtypes = [vp, vp, vp]
        L.chym_batch_get_shapes.argtypes = [vp, vp, vp, vp]
        L.chym_checkpoint.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_size_t), vp]
        L.chym_restore.argtypes = [vp, vp, ctypes.c_size_t, vp]
        L.chym_exit_scan_device.argtypes = [vp, vp, dbl, vp, ctypes.c_float, ctypes.c_int64,
                                            ctypes.c_int64, vp, vp, vp]
        L.chym_batch_set_shapes.argtypes = [vp, vp, vp, vp]
        L.chym_stats_noalloc.argtypes = [vp, i32, i32, i32, dbl, ctypes.POINTER(CStats), vp, vp,
                                         i32, vp]
        for name in EXPORTS:
            if name != "chym_last_error":
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise ChymError(status, lib().chym_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class Context:
    """One coupling matrix J and hyperspin dimension D; owns the device run state."""

    def __init__(self, J, D, kind=J_PM1):
        J = np.ascontiguousarray(J, dtype=np.float64)
        self.N = int(J.shape[0])
        self.D = int(D)
        self.kind = kind
        # the library's rule (uses_csr in chym_internal.cuh): a J with at most N^2 / 16
        # nonzeros runs its coupling product over the nonzeros on the CUDA cores in
        # FP32/FP64, and in BF16 hi+lo mode only for N >= 1024, D >= 3, on average at most
        # N / 256 nonzeros per row, and a run state (2 N D floats) within the SIMT
        # kernel's 200 KiB of shared memory
        self.nnz = int(np.count_nonzero(J))
        self.sparse = self.nnz * 16 <= self.N * self.N
        self.csr_bf16 = (self.sparse and self.N >= 1024 and self.D >= 3
                         and self.nnz * 256 <= self.N * self.N
                         and 2 * self.N * self.D * 4 <= 200 * 1024)
        h = ctypes.c_void_p()
        _check(lib().chym_create(_ptr(J), self.N, self.D, int(kind), ctypes.byref(h)))
        self._h = h

    def uses_csr(self, prec):
        """Whether steps at precision prec run the coupling over the nonzeros of J."""
        return self.sparse and (prec not in (PREC_BF16X2, PREC_FP8) or self.csr_bf16)

    def close(self):
        if getattr(self, "_h", None):
            lib().chym_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lambda_max(self):
        v = ctypes.c_double()
        _check(lib().chym_lambda_max(self._h, ctypes.byref(v)))
        return v.value

    def run(self, params: Params, h, seeds, steps, schedule: Schedule, stream=0, n_runs=None):
        """Host inputs: h (n_h), seeds (n_runs uint64) or None to continue."""
        h = None if h is None else np.ascontiguousarray(h, dtype=np.float64)
        if seeds is not None:
            seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
            n_runs = len(seeds)
        else:
            n_runs = n_runs if n_runs is not None else self.info()[0]
        n_h = len(h) if h is not None else self.info()[1]
        _check(lib().chym_run(self._h, ctypes.byref(params.c()), _ptr(h), n_h, _ptr(seeds),
                              n_runs, int(steps), ctypes.byref(schedule.c()),
                              ctypes.c_void_p(stream)))

    def run_device(self, params: Params, d_h, n_h, d_seeds, n_runs, steps, schedule: Schedule,
                   stream=0):
        """Device inputs: d_h / d_seeds are device addresses (int), d_seeds 0 to continue."""
        _check(lib().chym_run_device(self._h, ctypes.byref(params.c()), ctypes.c_void_p(d_h),
                                     int(n_h), ctypes.c_void_p(d_seeds), int(n_runs), int(steps),
                                     ctypes.byref(schedule.c()), ctypes.c_void_p(stream)))

    def checkpoint(self, stream=0):
        """The complete run state as bytes (chym_checkpoint)."""
        n = ctypes.c_size_t(0)
        _check(lib().chym_checkpoint(self._h, None, ctypes.byref(n), ctypes.c_void_p(stream)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().chym_checkpoint(self._h, buf, ctypes.byref(n), ctypes.c_void_p(stream)))
        return buf.raw[: n.value]

    def restore(self, data, stream=0):
        """Continue from bytes written by checkpoint() (chym_restore)."""
        _check(lib().chym_restore(self._h, data, len(data), ctypes.c_void_p(stream)))

    def info(self):
        n_runs, n_h, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().chym_info(self._h, ctypes.byref(n_runs), ctypes.byref(n_h), ctypes.byref(k)))
        return n_runs.value, n_h.value, k.value

    def energy(self, spins=False, stream=0):
        n_runs = self.info()[0]
        E = np.zeros(n_runs, dtype=np.float64)
        S = np.zeros((n_runs, (self.N + 63) // 64), dtype=np.uint64) if spins else None
        _check(lib().chym_energy(self._h, _ptr(E), _ptr(S), ctypes.c_void_p(stream)))
        return (E, S) if spins else E

    def energy_device(self, d_E, d_spins=0, stream=0):
        _check(lib().chym_energy_device(self._h, ctypes.c_void_p(d_E), ctypes.c_void_p(d_spins),
                                        ctypes.c_void_p(stream)))

    def set_coupling_weights(self, w=None):
        """Per-spin weights of the coupling term (chym_set_coupling_weights); None clears."""
        if w is None:
            _check(lib().chym_set_coupling_weights(self._h, None))
            return
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.shape == (self.N,)
        _check(lib().chym_set_coupling_weights(self._h, _ptr(w)))

    def energy_segments(self, seg_begin, stream=0):
        """Ising energies of the spin segments [seg_begin[i], seg_begin[i+1]):
        array [n_runs, n_seg] (chym_energy_segments)."""
        b = np.ascontiguousarray(seg_begin, dtype=np.int32)
        n_seg = len(b) - 1
        E = np.zeros((self.info()[0], n_seg), dtype=np.float64)
        _check(lib().chym_energy_segments(self._h, n_seg, _ptr(b), _ptr(E), ctypes.c_void_p(stream)))
        return E

    def readout_xy(self, spins=False, stream=0):
        """Best-axis rounding of D = 2 runs (chym_readout_xy): energies (and packed spins)."""
        n_runs = self.info()[0]
        E = np.zeros(n_runs, dtype=np.float64)
        S = np.zeros((n_runs, (self.N + 63) // 64), dtype=np.uint64) if spins else None
        _check(lib().chym_readout_xy(self._h, _ptr(E), _ptr(S), ctypes.c_void_p(stream)))
        return (E, S) if spins else E

    def readout_xy_device(self, d_E, d_spins=0, stream=0):
        _check(lib().chym_readout_xy_device(self._h, ctypes.c_void_p(d_E), ctypes.c_void_p(d_spins),
                                            ctypes.c_void_p(stream)))

    def stats(self, E_gs, n_bins=0, stream=0):
        n_runs, n_h, _ = self.info()
        st = CStats()
        hits = np.zeros(n_h, dtype=np.int64)
        hist = np.zeros(n_bins, dtype=np.int64) if n_bins else None
        _check(lib().chym_stats(self._h, float(E_gs), ctypes.byref(st), _ptr(hits), _ptr(hist),
                                int(n_bins), ctypes.c_void_p(stream)))
        out = {f: getattr(st, f) for f, _ in CStats._fields_}
        out["hits"] = hits
        if hist is not None:
            out["hist"] = hist
        return out

    def ground_state_exact(self):
        """Exact E_GS and minimiser (host, N <= 34)."""
        e = ctypes.c_double()
        S = np.zeros((1, (self.N + 63) // 64), dtype=np.uint64)
        _check(lib().chym_ground_state_exact(self._h, ctypes.byref(e), _ptr(S)))
        return e.value, unpack_spins(S, self.N)[0]

    def ground_state_search(self, restarts=32, sweeps=1000, seed=1):
        """Best-known E_GS by simulated annealing (host)."""
        e = ctypes.c_double()
        S = np.zeros((1, (self.N + 63) // 64), dtype=np.uint64)
        _check(lib().chym_ground_state_search(self._h, int(restarts), int(sweeps), int(seed),
                                              ctypes.byref(e), _ptr(S)))
        return e.value, unpack_spins(S, self.N)[0]

    def reseed_device(self, d_runs, n, d_new_seeds, init_std, d_new_pump=0, stream=0):
        """Restart the n runs listed at device address d_runs (int32) from new seeds,
        optionally with new pump indices (device int32)."""
        _check(lib().chym_reseed_device(self._h, ctypes.c_void_p(d_runs), int(n),
                                        ctypes.c_void_p(d_new_seeds), ctypes.c_void_p(d_new_pump),
                                        float(init_std), ctypes.c_void_p(stream)))

    def offsets_device(self, d_out, stream=0):
        _check(lib().chym_get_offsets_device(self._h, ctypes.c_void_p(d_out), ctypes.c_void_p(stream)))

    def exit_scan_device(self, d_E, E_gs, d_logits, theta, K, k_dec, d_counts, d_order, stream=0):
        """One decision pass of continuous operation (chym_exit_scan_device): device
        addresses d_E (float64), d_logits (float32 or 0), d_counts (int64[5]), d_order
        (int32[n_runs])."""
        _check(lib().chym_exit_scan_device(self._h, ctypes.c_void_p(d_E), float(E_gs),
                                           ctypes.c_void_p(d_logits or None), float(theta), int(K),
                                           int(k_dec), ctypes.c_void_p(d_counts),
                                           ctypes.c_void_p(d_order), ctypes.c_void_p(stream)))

    def copy_state_device(self, d_dst, stream=0):
        _check(lib().chym_copy_state_device(self._h, ctypes.c_void_p(d_dst), ctypes.c_void_p(stream)))

    def features_device(self, d_snapshot, k_frac, d_features, stream=0):
        _check(lib().chym_features_device(self._h, ctypes.c_void_p(d_snapshot), float(k_frac),
                                          ctypes.c_void_p(d_features), ctypes.c_void_p(stream)))

    def get_state(self, stream=0):
        n_runs, _, _ = self.info()
        X = np.zeros((n_runs, self.N, self.D), dtype=np.float64)
        k = ctypes.c_int64()
        _check(lib().chym_get_state(self._h, _ptr(X), ctypes.byref(k), ctypes.c_void_p(stream)))
        return X, k.value

    def set_state(self, X, h, seeds, k, prec, stream=0):
        X = np.ascontiguousarray(X, dtype=np.float64)
        h = np.ascontiguousarray(h, dtype=np.float64)
        seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        _check(lib().chym_set_state(self._h, _ptr(X), X.shape[0], _ptr(h), len(h), _ptr(seeds),
                                    int(k), int(prec), ctypes.c_void_p(stream)))


def ground_state_mobius(N, j_ring=-1.0, j_rung=-1.0):
    """Exact Ising ground-state energy of the Moebius ladder (host)."""
    e = ctypes.c_double()
    _check(lib().chym_ground_state_mobius(int(N), float(j_ring), float(j_rung), ctypes.byref(e)))
    return e.value


N_MLP_PARAMS = 5825
N_FEATURES = 24


class MLP:
    """The early-exit network (see chym_mlp_* in include/chym.h)."""

    def __init__(self, seed=1, max_batch=4096):
        h = ctypes.c_void_p()
        _check(lib().chym_mlp_create(int(seed), int(max_batch), ctypes.byref(h)))
        self._h = h

    def set_params(self, theta=None, mean=None, istd=None):
        f = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float32)
        theta, mean, istd = f(theta), f(mean), f(istd)
        _check(lib().chym_mlp_set_params(self._h, _ptr(theta), _ptr(mean), _ptr(istd)))

    def get_params(self):
        out = np.zeros(N_MLP_PARAMS, dtype=np.float32)
        _check(lib().chym_mlp_get_params(self._h, _ptr(out)))
        return out

    def forward_device(self, d_F, B, d_logits, stream=0):
        _check(lib().chym_mlp_forward_device(self._h, ctypes.c_void_p(d_F), int(B),
                                             ctypes.c_void_p(d_logits), ctypes.c_void_p(stream)))

    def grad_device(self, d_F, d_y, B, d_grad=0, d_loss=0, stream=0):
        _check(lib().chym_mlp_grad_device(self._h, ctypes.c_void_p(d_F), ctypes.c_void_p(d_y), int(B),
                                          ctypes.c_void_p(d_grad), ctypes.c_void_p(d_loss),
                                          ctypes.c_void_p(stream)))

    def train_step_device(self, d_F, d_y, B, lr, d_loss=0, stream=0):
        _check(lib().chym_mlp_train_step_device(self._h, ctypes.c_void_p(d_F), ctypes.c_void_p(d_y),
                                                int(B), float(lr), ctypes.c_void_p(d_loss),
                                                ctypes.c_void_p(stream)))

    def close(self):
        if getattr(self, "_h", None):
            lib().chym_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Several contexts integrated together (see chym_batch_* in include/chym.h)."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._h.value for c in self.contexts])
        h = ctypes.c_void_p()
        _check(lib().chym_batch_create(arr, len(self.contexts), ctypes.byref(h)))
        self._h = h

    def run(self, params, schedules, steps, stream=0):
        P = (CParams * len(self.contexts))(*[p.c() for p in params])
        S = (CSchedule * len(self.contexts))(*[s.c() for s in schedules])
        _check(lib().chym_batch_run(self._h, P, S, int(steps), ctypes.c_void_p(stream)))

    def status(self):
        _check(lib().chym_batch_status(self._h))

    def tuning(self):
        """The planner's cost model and tile shapes: {"chunk": [D=1..8], "k2": float,
        "tuned": bool, "shapes": {"rt": [...], "stages": [...], "ch": [...]}} (shape 0: the
        kernel's default)."""
        c = (ctypes.c_double * 8)()
        k2 = ctypes.c_double()
        t = ctypes.c_int32()
        _check(lib().chym_batch_get_tuning(self._h, c, ctypes.byref(k2), ctypes.byref(t)))
        return {"chunk": list(c), "k2": k2.value, "tuned": bool(t.value), "shapes": self.shapes()}

    def set_tuning(self, tuning):
        c = (ctypes.c_double * 8)(*tuning["chunk"])
        k2 = ctypes.c_double(tuning["k2"])
        _check(lib().chym_batch_set_tuning(self._h, c, ctypes.byref(k2)))
        if "shapes" in tuning:
            self.set_shapes(tuning["shapes"])

    def shapes(self):
        """Tile shapes per D = 1..8: large-N runs per column tile ("rt") and ring depth
        ("stages"), small-N epilogue chunk ("ch"); 0 stands for the kernel's default."""
        rt, st, ch = (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)()
        _check(lib().chym_batch_get_shapes(self._h, rt, st, ch))
        return {"rt": list(rt), "stages": list(st), "ch": list(ch)}

    def set_shapes(self, shapes):
        arr = [(ctypes.c_int32 * 8)(*shapes[k]) if k in shapes else None for k in ("rt", "stages", "ch")]
        _check(lib().chym_batch_set_shapes(self._h, *arr))

    def signature(self, device_key=""):
        """Key of the batch's composition for a tuning cache."""
        import hashlib
        parts = sorted((c.N, c.D, c.kind, c.info()[0]) for c in self.contexts)
        return hashlib.sha1(repr((device_key, parts)).encode()).hexdigest()[:16]

    def tune(self, params, schedules, probe_steps=64, stream=0, cache_path=None, device_key=""):
        """Measure the cost model (chym_batch_tune).  With cache_path, a JSON file of
        earlier tunings keyed by device_key and the batch's composition: a hit sets
        the cached costs without measuring, a miss measures and adds the entry."""
        import json
        import os
        key = self.signature(device_key)
        cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
            if key in cache:
                self.set_tuning(cache[key])
                return self.tuning()
        P = (CParams * len(self.contexts))(*[p.c() for p in params])
        S = (CSchedule * len(self.contexts))(*[s.c() for s in schedules])
        _check(lib().chym_batch_tune(self._h, P, S, int(probe_steps), ctypes.c_void_p(stream)))
        out = self.tuning()
        if cache_path:
            cache[key] = {"chunk": out["chunk"], "k2": out["k2"], "shapes": out["shapes"]}
            tmp = cache_path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(cache, f, indent=1, sort_keys=True)
            os.replace(tmp, cache_path)
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().chym_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stats_noalloc(d_E, n_runs, n_h, kind, E_gs, n_bins=0, stream=0, with_hits=True):
    """Figures of merit from device energies d_E (a device address) without any device
    allocation by the library (see chym_stats_noalloc in include/chym.h).  With
    with_hits=False no per-pump buffer is passed (the library then reads the counts it
    needs into its own host array) and the result has no "hits" entry."""
    st = CStats()
    hits = np.zeros(n_h, dtype=np.int64) if with_hits else None
    hist = np.zeros(n_bins, dtype=np.int64) if n_bins else None
    _check(lib().chym_stats_noalloc(ctypes.c_void_p(d_E), int(n_runs), int(n_h), int(kind),
                                    float(E_gs), ctypes.byref(st), _ptr(hits), _ptr(hist),
                                    int(n_bins), ctypes.c_void_p(stream)))
    out = {f: getattr(st, f) for f, _ in CStats._fields_}
    if hits is not None:
        out["hits"] = hits
    if hist is not None:
        out["hist"] = hist
    return out


def unpack_spins(words, N):
    """Bit-packed spins (bit p of word p // 64 set for +1) to an int8 array of +-1."""
    words = np.asarray(words, dtype=np.uint64)
    bits = np.unpackbits(words.view(np.uint8).reshape(words.shape[0], -1), axis=1,
                         bitorder="little")[:, :N]
    return (bits.astype(np.int8) * 2 - 1)
