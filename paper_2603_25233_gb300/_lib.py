"""ctypes declarations of the C ABI in include/rte.h (argument marshalling only).

The shared library is loaded from this package directory; there is no fallback: if it is
missing or fails to load, importing the binding raises.
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librte.so")

RTE_OK = 0
RTE_ERR_ARG = -1
RTE_ERR_CUDA = -2
RTE_ERR_NOMEM = -3
RTE_ERR_NOT_CONVERGED = -4
RTE_ERR_DEP_TIMEOUT = -5
RTE_ERR_SINGULAR = -6
RTE_ERR_NAN = -7
RTE_ERR_STATE = -8
RTE_FP64 = 0
RTE_FP32 = 1
RTE_DWF32 = 2
RTE_MODE_FR = 0
RTE_MODE_LR = 1

_ERR_NAMES = {v: k for k, v in dict(
    RTE_ERR_ARG=-1, RTE_ERR_CUDA=-2, RTE_ERR_NOMEM=-3, RTE_ERR_NOT_CONVERGED=-4,
    RTE_ERR_DEP_TIMEOUT=-5, RTE_ERR_SINGULAR=-6, RTE_ERR_NAN=-7, RTE_ERR_STATE=-8).items()}


class RteProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("x0", ctypes.c_double), ("x1", ctypes.c_double),
                ("y0", ctypes.c_double), ("y1", ctypes.c_double),
                ("n_theta", ctypes.c_int), ("n_omz", ctypes.c_int),
                ("sig_t", ctypes.POINTER(ctypes.c_double)),
                ("sig_s", ctypes.POINTER(ctypes.c_double)),
                ("q_cell", ctypes.POINTER(ctypes.c_double)),
                ("n_rect", ctypes.c_int),
                ("q_rects", ctypes.POINTER(ctypes.c_double)),
                ("inflow", ctypes.c_double * 4),
                ("n_gauss", ctypes.c_int),
                ("q_gauss", ctypes.POINTER(ctypes.c_double))]


class RteOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("sweep_precision", ctypes.c_int),
                ("eps_si", ctypes.c_double), ("eps_res", ctypes.c_double),
                ("eps_diff", ctypes.c_double), ("eps_svd", ctypes.c_double),
                ("eps_mgs", ctypes.c_double), ("eps_break", ctypes.c_double),
                ("dsa_tol", ctypes.c_double), ("dsa_max_iter", ctypes.c_int),
                ("use_dsa", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int),
                ("m_max", ctypes.c_int), ("mgs_test", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("truncate", ctypes.c_int), ("want_factors", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("sweep_refine", ctypes.c_int),
                ("dsa_precision", ctypes.c_int), ("basis_precision", ctypes.c_int),
                ("tc_projection", ctypes.c_int), ("sampling", ctypes.c_int),
                ("basis_update", ctypes.c_int)]


class RteStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("converged", ctypes.c_int),
                ("outer_iters", ctypes.c_int), ("total_inner", ctypes.c_int),
                ("total_sweeps", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("final_rank", ctypes.c_int), ("final_rank_trunc", ctypes.c_int),
                ("mgs_failures", ctypes.c_int), ("breakdowns", ctypes.c_int),
                ("full_checks", ctypes.c_int), ("dsa_cg_iters", ctypes.c_int),
                ("last_diff", ctypes.c_double), ("cell_angle_updates", ctypes.c_longlong),
                ("full_qr", ctypes.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


RTE_SWEEP_BAND, RTE_SWEEP_WARP = 1, 2


class RteSweepConfig(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("warps", ctypes.c_int), ("depth", ctypes.c_int),
                ("staged", ctypes.c_int), ("angles_per_block", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["kernel"] = {RTE_SWEEP_BAND: "band", RTE_SWEEP_WARP: "warp"}.get(self.kernel, self.kernel)
        return d


_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "rte_default_opts": (None, [ctypes.POINTER(RteOpts)]),
    "rte_last_error": (ctypes.c_char_p, []),
    "rte_setup": (ctypes.c_int, [ctypes.POINTER(RteProblem), _vp, ctypes.POINTER(_vp)]),
    "rte_destroy": (ctypes.c_int, [_vp]),
    "rte_set_materials": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "rte_get_sizes": (ctypes.c_int, [_vp, _ip, _ip, _ip]),
    "rte_set_wait_limit": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rte_inject_failure": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rte_get_quadrature": (ctypes.c_int, [_vp, _dp, _dp, _dp, _dp]),
    "rte_get_source": (ctypes.c_int, [_vp, _vp]),
    "rte_sweep": (ctypes.c_int, [_vp, _ip, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
    "rte_sweep_adjoint": (ctypes.c_int, [_vp, _ip, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]),
    "rte_sweep_tune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(RteSweepConfig)]),
    "rte_sweep_set_config": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(RteSweepConfig)]),
    "rte_sweep_get_config": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.POINTER(RteSweepConfig)]),
    "rte_si_dsa_solve": (ctypes.c_int, [_vp, ctypes.POINTER(RteOpts), _vp, ctypes.POINTER(RteStats)]),
    "rte_sweep_batch": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_ip), _ip, ctypes.c_int,
                                       ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp)]),
    "rte_si_dsa_solve_batch": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(RteOpts),
                                              ctypes.POINTER(_vp), ctypes.POINTER(RteStats)]),
    "rte_be_step": (ctypes.c_int, [_vp, ctypes.POINTER(RteOpts), ctypes.c_double, _vp, _vp, _vp,
                                   ctypes.POINTER(RteStats)]),
    "rte_get_lowrank_state": (ctypes.c_int, [_vp, _ip, _ip, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                             ctypes.POINTER(_vp), ctypes.POINTER(_vp)]),
    "rte_get_factors": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _ip]),
    "rte_adjoint_grad": (ctypes.c_int, [_vp, ctypes.POINTER(RteOpts), _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(RteStats)]),
    "rte_basis_project": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp, ctypes.c_int, _vp]),
    "rte_dsa_apply": (ctypes.c_int, [_vp, _vp, _vp]),
    "rte_dsa_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _ip]),
    "rte_dsa_solve_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, _vp, _vp, _vp, _vp, ctypes.c_double,
                                             ctypes.c_int, _ip, _vp]),
    "rte_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rte_profile_read": (ctypes.c_int, [_vp, ctypes.c_int, _dp, ctypes.POINTER(ctypes.c_longlong), _dp, _dp]),
}

PROF_CLASSES = {"sweep": 0, "dsa_cg": 1, "basis": 2, "galerkin": 3, "stencil": 4, "svd": 5, "basis_pass": 6,
                "basis_xc": 7, "basis_xt": 8, "basis_tc": 9}

_lib = None


def load(path=LIB_PATH):
    """Load librte.so (raises OSError if it is missing: the product path has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class RteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(rc):
    if rc != RTE_OK:
        raise RteError(rc, load().rte_last_error().decode())
    return rc
