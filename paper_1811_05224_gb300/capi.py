"""ctypes binding of libstbem (include/stbem.h), same names as the C ABI.

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device buffers are torch CUDA tensors (PyTorch is the memory
manager); their ``data_ptr()`` is passed through.  There is no CPU fallback:
``load()`` raises if the shared library is missing or cannot be opened.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstbem.so")

STBEM_OK = 0
STBEM_ERR_ARG = -1
STBEM_ERR_CUDA = -2
STBEM_ERR_NOMEM = -3
STBEM_ERR_NOCONV = -4
STBEM_ERR_BREAKDOWN = -5
STBEM_ERR_NAN = -6
STBEM_ERR_TIMEOUT = -7
STBEM_ERR_REDUCE = -8
OP_V, OP_K, OP_D = 0, 1, 2
F64, F32 = 0, 1

ERR_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_NOMEM", -4: "ERR_NOCONV",
             -5: "ERR_BREAKDOWN", -6: "ERR_NAN", -7: "ERR_TIMEOUT", -8: "ERR_REDUCE"}

EXPORTS = [
    "stbem_version", "stbem_launch_count", "stbem_create", "stbem_destroy", "stbem_last_error", "stbem_mesh_create",
    "stbem_mesh_destroy", "stbem_op_bytes", "stbem_assemble", "stbem_assemble_ops", "stbem_assemble_lags", "stbem_fft_operator_bytes", "stbem_fft_operator", "stbem_apply_fft_workspace_bytes", "stbem_apply_fft", "stbem_solve_fft_workspace_bytes", "stbem_solve_fft", "stbem_solve_batched_fft_workspace_bytes", "stbem_solve_batched_fft", "stbem_apply_workspace_bytes",
    "stbem_apply", "stbem_apply_noalloc", "stbem_rhs", "stbem_lumped_mass", "stbem_solve_workspace_bytes", "stbem_solve",
    "stbem_solve_mixed_workspace_bytes", "stbem_solve_mixed", "stbem_round_f32",
    "stbem_to_bf16", "stbem_apply_tc", "stbem_apply_tc_comp", "stbem_debug_tc_stall", "stbem_pipe_peaks", "stbem_bf16_split3", "stbem_apply_tc3_workspace_bytes",
    "stbem_apply_tc3", "stbem_rhs_g_batched", "stbem_half_mass_add", "stbem_solve_batched_workspace_bytes",
    "stbem_solve_batched", "stbem_solve_adjoint", "stbem_grad_workspace_bytes", "stbem_grad",
    "stbem_ragged_create", "stbem_ragged_destroy", "stbem_ragged_sizes", "stbem_ragged_offsets",
    "stbem_ragged_assemble", "stbem_ragged_lumped_mass", "stbem_ragged_apply_workspace_bytes", "stbem_ragged_apply",
    "stbem_ragged_tune", "stbem_ragged_tune_report", "stbem_ragged_rhs", "stbem_ragged_solve_workspace_bytes",
    "stbem_ragged_solve", "stbem_ragged_solve_mixed_workspace_bytes", "stbem_ragged_solve_mixed",
    "stbem_mixed_mass_inverse", "stbem_lag_shard", "stbem_assemble_lag_blocks", "stbem_apply_lags_workspace_bytes",
    "stbem_apply_lags", "stbem_solve_sharded_workspace_bytes", "stbem_solve_sharded",
    "stbem_mesh_create_graded", "stbem_nu_op_bytes", "stbem_nu_assemble", "stbem_nu_apply", "stbem_nu_rhs",
    "stbem_nu_lumped_mass", "stbem_nu_solve",
    "stbem_domain_create", "stbem_domain_destroy", "stbem_domain_info", "stbem_m0_bytes", "stbem_m0_assemble",
    "stbem_m0_apply_workspace_bytes", "stbem_m0_apply", "stbem_planewave_data", "stbem_evaluate",
    "stbem_exact_slices", "stbem_apply_tc_exact", "stbem_apply_exact_workspace_bytes", "stbem_apply_exact",
    "stbem_solve_batched_exact_workspace_bytes", "stbem_solve_batched_exact",
    "stbem_tune_cache_path", "stbem_tune_cache_get", "stbem_tune_cache_put", "stbem_tune_cache_clear", "stbem_tc_tune",
    "stbem_solve_mixed_exact_workspace_bytes", "stbem_solve_mixed_exact",
    "stbem_solve_mixed_tc_workspace_bytes", "stbem_solve_mixed_tc",
]


# int (*)(double* dev_buf, size_t n, void* user): the caller's all-reduce
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)


class Problem(ctypes.Structure):
    _fields_ = [("xy", ctypes.POINTER(ctypes.c_double)), ("n_x", ctypes.c_int), ("n_t", ctypes.c_int),
                ("T", ctypes.c_double), ("alpha", ctypes.c_double)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("restart", ctypes.c_int),
                ("precondition", ctypes.c_int)]


class ExactOperand(ctypes.Structure):
    _fields_ = [("n_slices", ctypes.c_int), ("slices", ctypes.c_void_p), ("row_exp", ctypes.c_void_p)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


class StbemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERR_NAMES.get(code, "?"), code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Open libstbem.so (built by ``paper_1811_05224_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libstbem.so not found at %s: run paper_1811_05224_gb300.build.build() "
                           "(the CUDA library is required; there is no CPU fallback)" % path)
    L = ctypes.CDLL(path)
    vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    P = ctypes.POINTER
    L.stbem_version.restype = ctypes.c_char_p
    L.stbem_launch_count.restype = ctypes.c_ulonglong
    L.stbem_create.argtypes = [P(vp), i, vp]
    L.stbem_destroy.argtypes = [vp]
    L.stbem_destroy.restype = None
    L.stbem_last_error.argtypes = [vp]
    L.stbem_last_error.restype = ctypes.c_char_p
    L.stbem_mesh_create.argtypes = [vp, P(d), i, d, i, d, P(vp)]
    L.stbem_mesh_destroy.argtypes = [vp]
    L.stbem_mesh_destroy.restype = None
    L.stbem_op_bytes.argtypes = [vp, i, i, P(sz)]
    L.stbem_assemble.argtypes = [vp, vp, i, i, vp]
    L.stbem_assemble_ops.argtypes = [vp, vp, i, i, i, vp, vp, vp]
    L.stbem_assemble_lags.argtypes = [vp, vp, i, i, i, i, vp]
    L.stbem_apply_workspace_bytes.argtypes = [i, i, i, i, P(sz)]
    L.stbem_apply.argtypes = [vp, i, i, i, i, vp, i, vp, vp, vp, sz]
    L.stbem_apply_noalloc.argtypes = [vp, i, i, i, i, vp, i, vp, vp]
    L.stbem_rhs.argtypes = [vp, vp, vp, d, d, vp, vp, vp, sz]
    L.stbem_lumped_mass.argtypes = [vp, vp, vp]
    L.stbem_solve_workspace_bytes.argtypes = [i, i, i, P(sz)]
    L.stbem_solve.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, P(SolveOpts), P(SolveInfo), vp, sz]
    L.stbem_solve_adjoint.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, P(SolveOpts), P(SolveInfo), vp, sz]
    L.stbem_fft_operator_bytes.argtypes = [i, i, P(i), P(sz)]
    L.stbem_fft_operator.argtypes = [vp, i, i, i, vp, vp]
    L.stbem_apply_fft_workspace_bytes.argtypes = [i, i, i, P(sz)]
    L.stbem_apply_fft.argtypes = [vp, i, i, i, i, vp, vp, vp, vp, sz]
    L.stbem_solve_fft_workspace_bytes.argtypes = [i, i, i, P(sz)]
    L.stbem_solve_fft.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, P(SolveOpts), P(SolveInfo), vp, sz]
    L.stbem_solve_batched_fft_workspace_bytes.argtypes = [i, i, i, i, P(sz)]
    L.stbem_solve_batched_fft.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, P(SolveOpts), d,
                                          P(SolveInfo), vp, sz]
    L.stbem_grad_workspace_bytes.argtypes = [i, i, P(sz)]
    L.stbem_mixed_mass_inverse.argtypes = [vp, vp, vp]
    L.stbem_grad.argtypes = [vp, vp, vp, d, d, vp, vp, vp, vp, vp, vp, sz]
    ll = ctypes.c_longlong
    L.stbem_ragged_create.argtypes = [vp, i, P(Problem), P(vp)]
    L.stbem_ragged_destroy.argtypes = [vp]
    L.stbem_ragged_destroy.restype = None
    L.stbem_ragged_sizes.argtypes = [vp, P(ll), P(ll), P(ll)]
    L.stbem_ragged_offsets.argtypes = [vp, P(ll), P(ll), P(ll)]
    L.stbem_ragged_assemble.argtypes = [vp, vp, i, i, vp]
    L.stbem_ragged_lumped_mass.argtypes = [vp, vp, vp]
    L.stbem_ragged_apply_workspace_bytes.argtypes = [vp, P(sz)]
    L.stbem_ragged_apply.argtypes = [vp, vp, i, vp, vp, vp, vp, sz]
    L.stbem_ragged_tune.argtypes = [vp, vp, i, vp, vp, vp, vp, sz, P(i), P(i)]
    L.stbem_ragged_tune_report.argtypes = [vp, i, P(i), P(i), P(ctypes.c_float), P(i), P(i)]
    L.stbem_tune_cache_path.argtypes = [ctypes.c_char_p]
    L.stbem_tune_cache_get.argtypes = [ctypes.c_char_p, ctypes.c_char_p, sz]
    L.stbem_tune_cache_put.argtypes = [ctypes.c_char_p, ctypes.c_char_p]
    L.stbem_tune_cache_clear.argtypes = []
    L.stbem_tc_tune.argtypes = [vp, i, i, vp, i, vp, vp, P(i), P(i)]
    L.stbem_ragged_rhs.argtypes = [vp, vp, i, vp, P(d), vp, vp, vp, sz]
    L.stbem_ragged_solve_workspace_bytes.argtypes = [vp, i, P(sz)]
    L.stbem_ragged_solve.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, P(SolveOpts), P(SolveInfo), vp, sz]
    L.stbem_ragged_solve_mixed_workspace_bytes.argtypes = [vp, i, P(sz)]
    L.stbem_ragged_solve_mixed.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, P(SolveOpts), d, P(SolveInfo), vp, sz]
    L.stbem_solve_mixed_workspace_bytes.argtypes = [i, i, i, P(sz)]
    L.stbem_solve_mixed.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, P(SolveOpts), d, P(SolveInfo), vp, sz]
    L.stbem_solve_mixed_exact_workspace_bytes.argtypes = [i, i, i, i, P(sz)]
    L.stbem_solve_mixed_tc_workspace_bytes.argtypes = [i, i, i, i, P(sz)]
    L.stbem_solve_mixed_tc.argtypes = [vp, i, i, P(ExactOperand), vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                       P(SolveOpts), d, P(SolveInfo), vp, sz]
    L.stbem_solve_mixed_exact.argtypes = [vp, i, i, P(ExactOperand), vp, vp, vp, vp, vp, P(SolveOpts), d,
                                          P(SolveInfo), vp, sz]
    L.stbem_round_f32.argtypes = [vp, sz, vp, vp]
    L.stbem_to_bf16.argtypes = [vp, i, sz, vp, vp]
    L.stbem_apply_tc.argtypes = [vp, i, i, vp, i, vp, vp]
    L.stbem_debug_tc_stall.argtypes = [i, ctypes.c_longlong]
    L.stbem_pipe_peaks.argtypes = [vp, P(d)]
    L.stbem_lag_shard.argtypes = [i, i, i, i, i, P(i), P(i)]
    L.stbem_mesh_create_graded.argtypes = [vp, P(d), i, P(d), i, d, P(vp)]
    L.stbem_nu_op_bytes.argtypes = [vp, P(sz)]
    L.stbem_nu_assemble.argtypes = [vp, vp, i, vp]
    L.stbem_nu_apply.argtypes = [vp, i, i, vp, vp, vp]
    L.stbem_nu_rhs.argtypes = [vp, vp, vp, d, d, vp, vp]
    L.stbem_nu_lumped_mass.argtypes = [vp, vp, vp]
    L.stbem_nu_solve.argtypes = [vp, i, i, vp, vp, vp, vp, vp, P(SolveOpts), P(SolveInfo), vp, sz]
    L.stbem_assemble_lag_blocks.argtypes = [vp, vp, i, i, i, i, vp]
    L.stbem_apply_lags_workspace_bytes.argtypes = [i, i, i, i, P(sz)]
    L.stbem_apply_lags.argtypes = [vp, i, i, i, i, i, i, vp, i, vp, vp, i, vp, sz]
    L.stbem_solve_sharded_workspace_bytes.argtypes = [i, i, i, P(sz)]
    L.stbem_solve_sharded.argtypes = [vp, i, i, i, vp, vp, i, P(i), ALLREDUCE_FN, vp, vp, vp, vp, P(SolveOpts),
                                      P(SolveInfo), vp, sz]
    L.stbem_apply_tc_comp.argtypes = [vp, i, i, vp, i, vp, vp, i]
    L.stbem_bf16_split3.argtypes = [vp, sz, vp, vp, vp, vp]
    L.stbem_apply_tc3_workspace_bytes.argtypes = [i, i, i, P(sz)]
    L.stbem_apply_tc3.argtypes = [vp, i, i, vp, vp, vp, i, vp, vp, vp, sz]
    L.stbem_rhs_g_batched.argtypes = [vp, vp, i, P(d), vp]
    L.stbem_half_mass_add.argtypes = [vp, vp, i, vp, vp]
    L.stbem_solve_batched_workspace_bytes.argtypes = [i, i, i, i, i, P(sz)]
    L.stbem_solve_batched.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, vp, vp, vp, P(SolveOpts), d, P(SolveInfo),
                                      vp, sz]
    L.stbem_exact_slices.argtypes = [vp, ctypes.c_longlong, i, i, vp, vp, vp]
    L.stbem_apply_tc_exact.argtypes = [vp, i, i, P(ExactOperand), i, P(ExactOperand), vp]
    L.stbem_apply_exact_workspace_bytes.argtypes = [i, i, i, i, P(sz)]
    L.stbem_apply_exact.argtypes = [vp, i, i, P(ExactOperand), i, vp, vp, vp, sz]
    L.stbem_solve_batched_exact_workspace_bytes.argtypes = [i, i, i, i, i, P(sz)]
    L.stbem_solve_batched_exact.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp, P(ExactOperand), vp, vp, P(SolveOpts),
                                            d, P(SolveInfo), vp, sz]
    L.stbem_domain_create.argtypes = [vp, vp, P(d), i, P(i), i, P(vp)]
    L.stbem_domain_destroy.argtypes = [vp]
    L.stbem_domain_destroy.restype = None
    L.stbem_domain_info.argtypes = [vp, P(i), P(i), P(i), P(i)]
    L.stbem_m0_bytes.argtypes = [vp, P(sz)]
    L.stbem_m0_assemble.argtypes = [vp, vp, vp]
    L.stbem_m0_apply_workspace_bytes.argtypes = [vp, P(sz)]
    L.stbem_m0_apply.argtypes = [vp, vp, i, vp, d, vp, vp, sz]
    L.stbem_planewave_data.argtypes = [vp, vp, d, vp, vp]
    L.stbem_evaluate.argtypes = [vp, vp, vp, i, vp, vp, vp, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("stbem_version", "stbem_launch_count", "stbem_destroy", "stbem_mesh_destroy", "stbem_last_error",
                        "stbem_domain_destroy"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def check(ctx, code):
    if code != STBEM_OK:
        msg = load().stbem_last_error(ctx).decode() if ctx else ""
        raise StbemError(code, msg)
    return code
