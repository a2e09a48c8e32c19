"""GB300 submatrix-method density matrix: thin Python binding of include/smx.h.

Every step of the computation runs in the CUDA library ``lib/libsmx.so``;
this module only marshals arguments (numpy arrays for host buffers, torch
CUDA tensors for device buffers and streams).  The binding raises if the
library is missing: there is no CPU fallback.

The names follow the C ABI: ``SubmatrixDensity`` owns one ``smx_ctx``.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (BF16, BOUND_MODEL_FEATURES, BOUND_MODEL_PARAMS, FN_DENSITY, FN_INV, FN_INV_SQRT, FN_SQRT,  # noqa: F401
                   FP16, FP16X3, FP64, FUNCTIONS, PRECISIONS, SmxError, Stats, check)


def _ptr(a):
    """Address of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


def dense_density_noalloc(h_dev, n: int, mu: float, d_dev, stream: int | None = None) -> None:
    """D = 1/2 (I - sign(H - mu I)) of one dense symmetric n x n matrix (n <= 256), no device allocation.

    For callers that cannot allocate device memory when they need the result
    (a plug-in whose host framework owns the device pool, a loop that must not
    enter the allocator).  ``h_dev`` and ``d_dev`` are caller-owned CUDA
    tensors (row-major doubles).  The library keeps its work matrices in one
    fixed device array shared by all calls: make the first call on a device
    before any stream capture, and do not let calls overlap on the GPU.  The
    call waits for its stream to return the status.
    """
    lib = _lib.load()
    check(lib.smx_dense_density_noalloc(_ptr(h_dev), int(n), float(mu), _ptr(d_dev), C.c_void_p(stream or 0)),
          "smx_dense_density_noalloc")


class SubmatrixDensity:
    """One library context: a block-sparse symmetric H and its density matrix.

    Parameters mirror ``smx_create``: block sizes, block-CSC column pointers
    and rows (full symmetric pattern), values (column-major blocks), and an
    optional CUDA stream handle (an int; ``torch.cuda.current_stream().cuda_stream``).
    """

    def __init__(self, block_size, col_ptr, row_idx, values, stream: int | None = None):
        lib = _lib.load()
        self._lib = lib
        self.block_size = np.ascontiguousarray(block_size, dtype=np.int32)
        self.col_ptr = np.ascontiguousarray(col_ptr, dtype=np.int64)
        self.row_idx = np.ascontiguousarray(row_idx, dtype=np.int32)
        vals = np.ascontiguousarray(values, dtype=np.float64)
        self.n_values = int(vals.shape[0])
        self.n_block_cols = int(self.block_size.shape[0])
        ctx = C.c_void_p()
        check(lib.smx_create(C.byref(ctx), self.n_block_cols, _ptr(self.block_size), _ptr(self.col_ptr),
                             _ptr(self.row_idx), _ptr(vals), C.c_void_p(stream or 0)), "smx_create")
        self._ctx = ctx

    @classmethod
    def from_system(cls, sysm, stream: int | None = None):
        """Context for a ``synth.BlockCSC``-like object (block_size, col_ptr, row_idx, values)."""
        return cls(sysm.block_size, sysm.col_ptr, sysm.row_idx, sysm.values, stream)

    def close(self):
        if getattr(self, "_ctx", None):
            self._lib.smx_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- settings -----------------------------------------------------------
    def set_values(self, values, on_device: bool = False):
        if on_device:
            check(self._lib.smx_set_values(self._ctx, _ptr(values), 1), "smx_set_values")
        else:
            v = np.ascontiguousarray(values, dtype=np.float64)
            check(self._lib.smx_set_values(self._ctx, _ptr(v), 0), "smx_set_values")

    def set_filter_threshold(self, eps: float):
        check(self._lib.smx_set_filter_threshold(self._ctx, float(eps)), "smx_set_filter_threshold")

    def set_staging_limit(self, nbytes: int):
        check(self._lib.smx_set_staging_limit(self._ctx, C.c_uint64(int(nbytes))), "smx_set_staging_limit")

    def set_column_range(self, j0: int, j1: int):
        check(self._lib.smx_set_column_range(self._ctx, int(j0), int(j1)), "smx_set_column_range")

    def get_gershgorin_interval(self):
        lo, hi = C.c_double(0.0), C.c_double(0.0)
        check(self._lib.smx_get_gershgorin_interval(self._ctx, C.byref(lo), C.byref(hi)), "smx_get_gershgorin_interval")
        return lo.value, hi.value

    def set_mu(self, mu: float):
        check(self._lib.smx_set_mu(self._ctx, float(mu)), "smx_set_mu")

    def set_electron_count(self, n_e: float, max_steps: int = 30, tol: float = 0.5):
        check(self._lib.smx_set_electron_count(self._ctx, float(n_e), int(max_steps), float(tol)),
              "smx_set_electron_count")

    def set_precision(self, bulk="fp64", fp64_final_iters: int = 0):
        p = PRECISIONS[bulk] if isinstance(bulk, str) else int(bulk)
        check(self._lib.smx_set_precision(self._ctx, p, int(fp64_final_iters)), "smx_set_precision")

    def set_function(self, f="density"):
        """Matrix function of the following builds: "density" (default), "inv_sqrt", "sqrt", "inv" or
        "fermi" (FP64 form; see smx_set_function and smx_set_fermi_beta)."""
        check(self._lib.smx_set_function(self._ctx, FUNCTIONS[f] if isinstance(f, str) else int(f)),
              "smx_set_function")

    def set_fermi_beta(self, beta: float):
        """Inverse temperature of the "fermi" function form (smx_set_fermi_beta)."""
        check(self._lib.smx_set_fermi_beta(self._ctx, float(beta)), "smx_set_fermi_beta")

    def set_symmetrize(self, enable: bool = True):
        """Return 1/2 (D + D^T) on the filtered pattern from later builds (smx_set_symmetrize)."""
        check(self._lib.smx_set_symmetrize(self._ctx, 1 if enable else 0), "smx_set_symmetrize")

    def set_overlap(self, values=None, on_device: bool = False):
        """Overlap S on the input pattern (non-orthogonal form of Eq. 14; see smx_set_overlap);
        None returns to S = I."""
        if values is None:
            check(self._lib.smx_set_overlap(self._ctx, None, 0), "smx_set_overlap")
        elif on_device:
            check(self._lib.smx_set_overlap(self._ctx, _ptr(values), 1), "smx_set_overlap")
        else:
            v = np.ascontiguousarray(values, dtype=np.float64)
            check(self._lib.smx_set_overlap(self._ctx, _ptr(v), 0), "smx_set_overlap")

    # -- work ---------------------------------------------------------------
    def build_density(self):
        check(self._lib.smx_build_density(self._ctx), "smx_build_density")

    def solve_mu(self):
        check(self._lib.smx_solve_mu(self._ctx), "smx_solve_mu")

    def solve_mu_device(self):
        """The bisection with its decisions on the device (smx_solve_mu_device)."""
        check(self._lib.smx_solve_mu_device(self._ctx), "smx_solve_mu_device")

    # -- results ------------------------------------------------------------
    def get_trace(self):
        tr, en, mu = C.c_double(), C.c_double(), C.c_double()
        check(self._lib.smx_get_trace(self._ctx, C.byref(tr), C.byref(en), C.byref(mu)), "smx_get_trace")
        return tr.value, en.value, mu.value

    def get_density(self, out=None):
        """D laid out like the input values: into ``out`` (numpy or CUDA tensor) or a new numpy array."""
        if out is None:
            out = np.empty(self.n_values, dtype=np.float64)
        on_device = not isinstance(out, np.ndarray)
        check(self._lib.smx_get_density(self._ctx, _ptr(out), 1 if on_device else 0), "smx_get_density")
        return out

    def get_pattern(self):
        st = self.get_stats()
        cp = np.empty(self.n_block_cols + 1, dtype=np.int64)
        ri = np.empty(max(1, st["nnzb_filtered"]), dtype=np.int32)
        check(self._lib.smx_get_pattern(self._ctx, _ptr(cp), _ptr(ri)), "smx_get_pattern")
        return cp, ri[: st["nnzb_filtered"]]

    def get_stats(self) -> dict:
        s = Stats()
        check(self._lib.smx_get_stats(self._ctx, C.byref(s)), "smx_get_stats")
        return s.as_dict()

    def selftest_wait_timeout(self, poll_limit: int = 1 << 16) -> int:
        """Runs the bounded-wait self-test (smx_selftest_wait_timeout); returns its status code
        (ERR_TIMEOUT when the wait gave up as designed) without raising."""
        return int(self._lib.smx_selftest_wait_timeout(self._ctx, C.c_uint32(int(poll_limit))))

    def reset_counters(self):
        check(self._lib.smx_reset_counters(self._ctx), "smx_reset_counters")

    def get_submatrix_info(self):
        dims = np.empty(self.n_block_cols, dtype=np.int32)
        iters = np.empty(self.n_block_cols, dtype=np.int32)
        bounds = np.empty(self.n_block_cols, dtype=np.float64)
        check(self._lib.smx_get_submatrix_info(self._ctx, _ptr(dims), _ptr(iters), _ptr(bounds)),
              "smx_get_submatrix_info")
        return dims, iters, bounds

    # learned spectral bound -------------------------------------------------

    def bound_model_init(self, seed: int = 0):
        check(self._lib.smx_bound_model_init(self._ctx, C.c_uint64(seed)), "smx_bound_model_init")

    def bound_model_set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        check(self._lib.smx_bound_model_set_params(self._ctx, _ptr(p), int(p.shape[0])), "smx_bound_model_set_params")

    def bound_model_get_params(self):
        p = np.empty(BOUND_MODEL_PARAMS, dtype=np.float32)
        check(self._lib.smx_bound_model_get_params(self._ctx, _ptr(p), BOUND_MODEL_PARAMS), "smx_bound_model_get_params")
        return p

    def bound_model_collect(self, lanczos_steps: int = 48):
        check(self._lib.smx_bound_model_collect(self._ctx, int(lanczos_steps)), "smx_bound_model_collect")

    def bound_model_train(self, epochs: int, batch: int = 256, lr: float = 1e-3) -> float:
        loss = C.c_double(0.0)
        check(self._lib.smx_bound_model_train(self._ctx, int(epochs), int(batch), float(lr), C.byref(loss)),
              "smx_bound_model_train")
        return loss.value

    def bound_model_fit(self, x, t, steps: int = 0, lr: float = 1e-3):
        """Loss and gradient at the current parameters on (x [m, 9], t [m, 2]), then ``steps`` Adam steps."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        assert x.ndim == 2 and x.shape[1] == BOUND_MODEL_FEATURES and t.shape == (x.shape[0], 2)
        g = np.empty(BOUND_MODEL_PARAMS, dtype=np.float32)
        loss = C.c_double(0.0)
        check(self._lib.smx_bound_model_fit(self._ctx, _ptr(x), _ptr(t), int(x.shape[0]), int(steps), float(lr),
                                            _ptr(g), C.byref(loss)), "smx_bound_model_fit")
        return loss.value, g

    def bound_model_predict(self, predict: bool = True, labels: bool = False, lanczos_steps: int = 48):
        """(features [B, 9], predictions [B, 2] or None, Lanczos labels [B, 2] or None) at the fixed mu."""
        f = np.empty((self.n_block_cols, BOUND_MODEL_FEATURES), dtype=np.float32)
        p = np.empty((self.n_block_cols, 2), dtype=np.float32) if predict else None
        lab = np.empty((self.n_block_cols, 2), dtype=np.float32) if labels else None
        check(self._lib.smx_bound_model_predict(self._ctx, _ptr(f), _ptr(p) if p is not None else None,
                                                _ptr(lab) if lab is not None else None, int(lanczos_steps)),
              "smx_bound_model_predict")
        return f, p, lab

    def set_bound_model(self, enable=True, weights_path: str | None = None):
        """enable: False / "off" (0), True / "gap" (1: rho_hat and the gap-driven scaled
        schedule) or "rho" (2: rho_hat only); see smx_set_bound_model."""
        modes = {"off": 0, "gap": 1, "rho": 2}
        mode = modes[enable] if isinstance(enable, str) else int(enable)
        path = weights_path.encode() if weights_path is not None else None
        check(self._lib.smx_set_bound_model(self._ctx, mode, path), "smx_set_bound_model")

    def bound_model_save(self, path: str):
        check(self._lib.smx_bound_model_save(self._ctx, path.encode()), "smx_bound_model_save")
