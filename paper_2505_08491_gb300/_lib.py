"""ctypes declarations of the md C ABI (include/md.h).  Marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmd_gb300.so")

MD_OK, MD_NOT_CONVERGED = 0, 1
STATUS_NAMES = {0: "MD_OK", 1: "MD_NOT_CONVERGED", -1: "MD_ERR_ARG", -2: "MD_ERR_OOM", -3: "MD_ERR_CUDA",
                -4: "MD_ERR_TIMEOUT", -5: "MD_ERR_NAN", -6: "MD_ERR_IO", -7: "MD_ERR_UNIMPLEMENTED"}
MD_FP32, MD_FP64 = 0, 1
MD_SOLVER_FGMRES_CNN, MD_SOLVER_FGMRES_JACOBI, MD_SOLVER_CG_JACOBI = 0, 1, 2
MD_CNN_NPARAMS = 114209


class MdGraph(C.Structure):
    _fields_ = [("n_nodes", C.c_int), ("xyz", C.POINTER(C.c_double)), ("n_edges", C.c_int),
                ("edges", C.POINTER(C.c_int)), ("elems_per_edge", C.c_int)]


class MdParams(C.Structure):
    _fields_ = [("k_omega", C.c_double), ("sigma_omega", C.c_double), ("k_lambda", C.c_double),
                ("natural_boundary", C.c_int), ("n_dirichlet_1d", C.c_int), ("dirichlet_1d", C.POINTER(C.c_int)),
                ("u_d", C.c_double)]


class MdOpInfo(C.Structure):
    _fields_ = [("N", C.c_int), ("n3", C.c_int), ("n1", C.c_int), ("nq", C.c_int), ("n_touch", C.c_int),
                ("n", C.c_longlong), ("alpha", C.c_double), ("beta", C.c_double)]


class MdBatchStats(C.Structure):
    _fields_ = [("kernel_launches", C.c_longlong), ("cycles", C.c_longlong), ("iterations", C.c_longlong),
                ("precond_nodes", C.c_longlong), ("prec_ms", C.c_double), ("conv_hidden_ms", C.c_double),
                ("conv_hidden_launches", C.c_longlong), ("apply_ms", C.c_double), ("arnoldi_ms", C.c_double),
                ("restart_ms", C.c_double), ("fallback_instances", C.c_longlong), ("graph_launches", C.c_longlong),
                ("slot_gating", C.c_longlong)]


class MdTuning(C.Structure):
    _fields_ = [("tuned", C.c_int), ("vec_chunk", C.c_int), ("n_vec", C.c_int), ("vec_candidates", C.c_int * 8),
                ("vec_us", C.c_double * 8), ("conv_tps", C.c_int), ("conv_us", C.c_double * 2)]


class MdTrainCfg(C.Structure):
    _fields_ = [("n_ops", C.c_int), ("ops", C.POINTER(C.c_void_p)), ("n_samples", C.c_int),
                ("sample_op", C.POINTER(C.c_int)), ("sample_r", C.POINTER(C.c_void_p)),
                ("epochs", C.c_int), ("batch", C.c_int),
                ("lr", C.c_double), ("lr_min", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("weight_decay", C.c_double), ("eps", C.c_double), ("seed", C.c_uint64),
                ("loss_history", C.POINTER(C.c_double))]


vp = C.c_void_p
i32 = C.c_int
i64 = C.c_longlong
f64 = C.c_double
st = C.c_int

# name: (restype, argtypes)
SIGNATURES = {
    "md_assemble": (st, [i32, C.POINTER(MdGraph), f64, f64, C.POINTER(MdParams), C.POINTER(vp)]),
    "md_op_destroy": (None, [vp]),
    "md_op_get_info": (st, [vp, C.POINTER(MdOpInfo)]),
    "md_op_distance": (st, [vp, vp, vp]),
    "md_rhs": (st, [vp, vp, f64, vp, vp]),
    "md_apply": (st, [vp, i32, vp, vp, vp]),
    "md_apply_noalloc": (st, [vp, i32, vp, vp, vp]),
    "md_cnn_create": (st, [C.POINTER(C.c_float), i64, C.POINTER(vp)]),
    "md_cnn_get_params": (st, [vp, C.POINTER(C.c_float), i64]),
    "md_cnn_set_engine": (st, [vp, i32]),
    "md_cnn_destroy": (None, [vp]),
    "md_cnn_save": (st, [vp, C.c_char_p]),
    "md_cnn_load": (st, [C.c_char_p, C.POINTER(vp)]),
    "md_cnn_forward": (st, [vp, i32, i32, vp, vp, vp]),
    "md_unet_num_params": (i64, []),
    "md_unet_create": (st, [C.POINTER(C.c_float), i64, C.POINTER(vp)]),
    "md_unet_destroy": (None, [vp]),
    "md_unet_forward": (st, [vp, i32, i32, vp, vp, vp]),
    "md_unet_backward": (st, [vp, i32, i32, vp, vp, vp, vp, vp]),
    "md_unet_set_params": (st, [vp, vp, i32, vp]),
    "md_unet_get_params": (st, [vp, C.POINTER(C.c_float), i64]),
    "md_unet_train_loss": (st, [vp, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(f64), vp, vp]),
    "md_unet_opt_step": (st, [vp, vp, f64, f64, f64, f64, f64, vp]),
    "md_batch_set_unet": (st, [vp, vp]),
    "md_cnn_backward": (st, [vp, i32, i32, vp, vp, vp, vp, vp]),
    "md_precondition": (st, [vp, vp, vp, vp, vp]),
    "md_lift": (st, [vp, vp, vp, vp, vp]),
    "md_precondition_lower": (st, [vp, vp, vp, vp, vp]),
    "md_batch_set_prec_order": (st, [vp, i32]),
    "md_batch_set_smoothing": (st, [vp, i32, f64]),
    "md_precondition_smoothed": (st, [vp, vp, i32, i32, f64, vp, vp, vp]),
    "md_batch_set_inner_iters": (st, [vp, i32]),
    "md_precondition_inner": (st, [vp, vp, i32, i32, vp, vp, vp]),
    "md_solve": (st, [vp, vp, vp, vp, f64, i32, i32, C.POINTER(i32), C.POINTER(f64), vp]),
    "md_batch_create": (st, [i32, C.POINTER(vp), vp, i32, i32, C.POINTER(vp)]),
    "md_batch_destroy": (None, [vp]),
    "md_batch_offsets": (st, [vp, C.POINTER(i64)]),
    "md_batch_solve": (st, [vp, vp, vp, f64, i32, C.POINTER(i32), C.POINTER(f64), vp]),
    "md_batch_times": (st, [vp, C.POINTER(f64)]),
    "md_batch_set_profiling": (st, [vp, i32]),
    "md_batch_set_host_loop": (st, [vp, i32]),
    "md_batch_tuning": (st, [vp, C.POINTER(MdTuning)]),
    "md_batch_stats": (st, [vp, C.POINTER(MdBatchStats)]),
    "md_batch_reset_stats": (st, [vp]),
    "md_solve_batched": (st, [i32, C.POINTER(vp), vp, C.POINTER(vp), C.POINTER(vp), f64, i32, i32,
                              C.POINTER(i32), C.POINTER(f64), vp]),
    "md_train": (st, [vp, C.POINTER(MdTrainCfg)]),
    "md_train_loss": (st, [vp, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(f64), vp, vp]),
    "md_krylov_basis": (st, [vp, vp, i32, vp, vp]),
    "md_opt_create": (st, [vp, C.POINTER(vp)]),
    "md_opt_step": (st, [vp, vp, vp, f64, f64, f64, f64, f64, vp]),
    "md_opt_destroy": (None, [vp]),
    "md_last_error": (C.c_char_p, []),
    "md_version": (C.c_char_p, []),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library and declare every entry point.  Raises if the
    library has not been built: there is no fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"md library not built: {path} is missing "
                           "(run python -m paper_2505_08491_gb300.build)")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class MdError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def check(status: int, where: str, allow=(MD_OK,)):
    if status not in allow:
        raise MdError(status, where, load().md_last_error().decode(errors="replace"))
    return status
