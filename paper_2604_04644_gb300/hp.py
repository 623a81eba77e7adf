"""ctypes binding of the libhp C ABI (include/hp.h): same names, argument
marshalling only.  Every operator runs in the library's CUDA kernels; if the
shared library is missing this module raises at import time.

Device arrays are passed as torch CUDA tensors (or raw integer addresses);
streams as torch.cuda.Stream, an integer cudaStream_t, or None for the
current torch stream.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhp.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libhp.so is not built (run __graft_entry__.build() or "
                      "python -m paper_2604_04644_gb300.build); there is no fallback path")
_lib = ctypes.CDLL(LIB_PATH)

# enums (values from include/hp.h)
HP_OK, HP_ERR_ARG, HP_ERR_OOM, HP_ERR_CUDA, HP_ERR_GEOM, HP_ERR_UNSUPPORTED, HP_ERR_TIMEOUT, \
    HP_ERR_DEVICE_BOUNDS, HP_ERR_NOT_CONVERGED = range(9)
HP_HEX, HP_PRISM, HP_PYR, HP_TET = range(4)
HP_MASS, HP_LAPLACIAN, HP_HELMHOLTZ, HP_BWDTRANS, HP_IPRODUCT_WRT_BASE, HP_PHYSDERIV, \
    HP_IPRODUCT_WRT_DERIV_BASE, HP_ADVECTION_DIFFUSION_REACTION = range(8)
HP_STRAT_SUMFAC, HP_STRAT_ELEMAT, HP_STRAT_HYBRID, HP_STRAT_AUTO = range(4)
HP_STRAT_MATRIX = 4
HP_FP64, HP_FP32, HP_TF32, HP_BF16 = range(4)

EXPORTED = ["hp_mesh_create", "hp_mesh_layout", "hp_geom_factors", "hp_geom_copy", "hp_op_create",
            "hp_op_apply", "hp_op_apply_graph", "hp_op_tune", "hp_op_tiles", "hp_op_strategies",
            "hp_op_set_collocated", "hp_op_set_deterministic", "hp_op_set_advection", "hp_op_set_batching", "hp_op_block_features", "hp_op_schedule", "hp_op_schedule_mlp", "hp_op_schedule_exhaustive",
            "hp_op_schedule_graph", "hp_op_sync", "hp_op_work",
            "hp_op_block_work", "hp_op_apply_block", "hp_peak_fp64",
            "hp_op_destroy", "hp_mesh_destroy", "hp_status_str", "hp_last_error",
            "hp_mlp_create", "hp_mlp_info", "hp_mlp_params", "hp_mlp_forward", "hp_mlp_grad", "hp_mlp_adam_step",
            "hp_mlp_destroy", "hp_mlp_grad_noalloc", "hp_mesh_points", "hp_c0_create", "hp_c0_info",
            "hp_c0_map_host", "hp_c0_maps", "hp_c0_gather", "hp_c0_assemble", "hp_solve", "hp_c0_destroy", "hp_c0_diagonal",
            "hp_partition", "hp_halo_create", "hp_halo_info", "hp_halo_counts", "hp_halo_maps", "hp_halo_gather",
            "hp_halo_reduce_pack", "hp_halo_reduce_sum", "hp_halo_bcast_pack", "hp_halo_bcast_unpack",
            "hp_halo_destroy", "hp_xdot_acc", "hp_xacc_round", "hp_xacc_limbs",
            "hp_mesh2d_create", "hp_mesh2d_layout", "hp_op2d_apply", "hp_mesh2d_factors", "hp_mesh2d_sync",
            "hp_mesh2d_destroy"]


class HpError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.hp_last_error().decode()
        super().__init__("%s failed: %s (%s)" % (where, _lib.hp_status_str(status).decode(), msg))


class hp_mesh_desc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("shape", ctypes.c_void_p), ("P", ctypes.c_void_p),
                ("Q", ctypes.c_void_p), ("vert", ctypes.c_void_p), ("xyz", ctypes.c_void_p),
                ("n_vert", ctypes.c_int64), ("curved", ctypes.c_void_p), ("deformation", ctypes.c_int32),
                ("geometry", ctypes.c_int32), ("quadrature", ctypes.c_int32)]


class hp_mesh2d_desc(ctypes.Structure):
    _fields_ = [("n_elem", ctypes.c_int64), ("shape", ctypes.c_void_p), ("P", ctypes.c_void_p),
                ("vert", ctypes.c_void_p), ("xy", ctypes.c_void_p), ("n_vert", ctypes.c_int64),
                ("curved", ctypes.c_void_p), ("deformation", ctypes.c_int32)]


_vp, _i64p, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
_lib.hp_mesh_create.argtypes = [ctypes.POINTER(hp_mesh_desc), ctypes.c_int, ctypes.POINTER(_vp)]
_lib.hp_mesh_layout.argtypes = [_vp, _vp, _vp, _i64p, _i64p]
_lib.hp_geom_factors.argtypes = [_vp, _vp]
_lib.hp_geom_copy.argtypes = [_vp, _vp, _vp]
_lib.hp_op_create.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]
_lib.hp_op_apply.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp]
_lib.hp_op_apply_graph.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp]
_lib.hp_op_tune.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp]
_lib.hp_op_tiles.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int]
_lib.hp_op_strategies.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int]
_lib.hp_op_set_collocated.argtypes = [_vp, ctypes.c_int]
_lib.hp_op_set_deterministic.argtypes = [_vp, ctypes.c_int]
_lib.hp_op_set_advection.argtypes = [_vp, _vp]
_lib.hp_op_set_batching.argtypes = [_vp, ctypes.c_int]
_lib.hp_op_set_batching.restype = ctypes.c_int
_lib.hp_op_set_advection.restype = ctypes.c_int
_lib.hp_op_set_deterministic.restype = ctypes.c_int
_lib.hp_op_block_features.argtypes = [_vp, _vp, ctypes.c_int64]
_lib.hp_op_schedule.argtypes = [_vp, _vp, _vp]
_lib.hp_op_schedule_mlp.argtypes = [_vp, _vp, ctypes.c_int, _vp]
_lib.hp_op_schedule_mlp.restype = ctypes.c_int
_lib.hp_op_schedule_exhaustive.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp, _vp]
_lib.hp_op_schedule_graph.argtypes = [_vp, ctypes.c_double, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.hp_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                               ctypes.POINTER(_vp)]
_lib.hp_mlp_info.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.hp_mlp_params.argtypes = [_vp, _vp, ctypes.c_int64, ctypes.c_int]
_lib.hp_mlp_forward.argtypes = [_vp, _vp, ctypes.c_int64, _vp, _vp]
_lib.hp_mlp_grad.argtypes = [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]
_lib.hp_mlp_adam_step.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_float, _vp, _vp]
_lib.hp_mlp_destroy.argtypes = [_vp]
_lib.hp_mlp_grad_noalloc.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, ctypes.c_int64, _vp,
                                     _vp, _vp]
_lib.hp_mlp_grad_noalloc.restype = ctypes.c_int
_lib.hp_op_sync.argtypes = [_vp, _vp]
_lib.hp_op_work.argtypes = [_vp, _i64p, _dp, _dp]
_lib.hp_op_block_work.argtypes = [_vp, ctypes.c_int64, _i64p, _i64p, _dp, _dp, _dp]
_lib.hp_op_apply_block.argtypes = [_vp, ctypes.c_int64, ctypes.c_double, _vp, _vp, _vp]
_lib.hp_peak_fp64.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _vp]
_lib.hp_peak_fp64.restype = ctypes.c_int
_lib.hp_op_destroy.argtypes = [_vp]
_lib.hp_mesh2d_create.argtypes = [ctypes.POINTER(hp_mesh2d_desc), ctypes.c_int, ctypes.POINTER(_vp)]
_lib.hp_mesh2d_layout.argtypes = [_vp, _vp, _vp]
_lib.hp_op2d_apply.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _vp, _vp, _vp]
_lib.hp_mesh2d_factors.argtypes = [_vp, _vp]
_lib.hp_mesh2d_sync.argtypes = [_vp, _vp]
_lib.hp_mesh2d_destroy.argtypes = [_vp]
_lib.hp_mesh2d_destroy.restype = None
_lib.hp_mesh_destroy.argtypes = [_vp]
_lib.hp_status_str.argtypes = [ctypes.c_int]
_lib.hp_status_str.restype = ctypes.c_char_p
_lib.hp_last_error.restype = ctypes.c_char_p
for _f in ("hp_mesh_create", "hp_mesh_layout", "hp_geom_factors", "hp_geom_copy", "hp_op_create",
           "hp_op_apply", "hp_op_apply_graph", "hp_op_tune", "hp_op_tiles", "hp_op_sync", "hp_op_work",
           "hp_op_block_work", "hp_op_apply_block", "hp_op_strategies", "hp_op_set_collocated", "hp_op_set_deterministic", "hp_op_set_advection", "hp_op_set_batching", "hp_op_block_features", "hp_op_schedule", "hp_op_schedule_exhaustive",
           "hp_op_schedule_graph", "hp_mlp_create", "hp_mlp_info", "hp_mlp_params", "hp_mlp_forward", "hp_mlp_grad", "hp_mlp_adam_step"):
    getattr(_lib, _f).restype = ctypes.c_int


def _check(st, where):
    if st != HP_OK:
        raise HpError(st, where)


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError("cannot take the address of %r" % type(x))


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def hp_mesh_create(mesh, device=0):
    """mesh: dict with the hp_mesh_desc arrays (see paper_2604_04644_gb300.inputs)."""
    keep = dict(
        shape=np.ascontiguousarray(mesh["shape"], dtype=np.uint8),
        P=np.ascontiguousarray(mesh["P"], dtype=np.uint8),
        Q=np.ascontiguousarray(mesh["Q"], dtype=np.uint8),
        vert=np.ascontiguousarray(mesh["vert"], dtype=np.int64),
        xyz=np.ascontiguousarray(mesh["xyz"], dtype=np.float64),
        curved=np.ascontiguousarray(mesh["curved"], dtype=np.uint8),
    )
    d = hp_mesh_desc(int(mesh["n_elem"]), keep["shape"].ctypes.data, keep["P"].ctypes.data,
                     keep["Q"].ctypes.data, keep["vert"].ctypes.data, keep["xyz"].ctypes.data,
                     int(keep["xyz"].shape[0]), keep["curved"].ctypes.data, int(mesh["deformation"]),
                     int(mesh.get("geometry", 0)), int(mesh.get("quadrature", 0)))
    h = _vp()
    _check(_lib.hp_mesh_create(ctypes.byref(d), int(device), ctypes.byref(h)), "hp_mesh_create")
    return h.value


HP_QUAD, HP_TRI = 4, 5


def hp_mesh2d_create(mesh, device=0):
    """mesh: dict with the hp_mesh2d_desc arrays (see inputs.square_mesh_2d)."""
    keep = dict(shape=np.ascontiguousarray(mesh["shape"], dtype=np.uint8),
                P=np.ascontiguousarray(mesh["P"], dtype=np.uint8),
                vert=np.ascontiguousarray(mesh["vert"], dtype=np.int64),
                xy=np.ascontiguousarray(mesh["xy"], dtype=np.float64),
                curved=np.ascontiguousarray(mesh["curved"], dtype=np.uint8))
    d = hp_mesh2d_desc(int(mesh["n_elem"]), keep["shape"].ctypes.data, keep["P"].ctypes.data, keep["vert"].ctypes.data,
                       keep["xy"].ctypes.data, int(keep["xy"].shape[0]), keep["curved"].ctypes.data,
                       int(mesh["deformation"]))
    h = _vp()
    _check(_lib.hp_mesh2d_create(ctypes.byref(d), int(device), ctypes.byref(h)), "hp_mesh2d_create")
    return h.value


def hp_mesh2d_layout(mesh, n_elem):
    co = np.zeros(n_elem + 1, dtype=np.int64)
    po = np.zeros(n_elem + 1, dtype=np.int64)
    _check(_lib.hp_mesh2d_layout(mesh, co.ctypes.data, po.ctypes.data), "hp_mesh2d_layout")
    return co, po


def hp_op2d_apply(mesh, kind, dtype, lam, x, y, stream=None):
    _check(_lib.hp_op2d_apply(mesh, int(kind), int(dtype), float(lam), _ptr(x), _ptr(y), _stream(stream)),
           "hp_op2d_apply")


def hp_mesh2d_factors(mesh, n_phys):
    out = np.zeros(4 * int(n_phys), dtype=np.float64)
    _check(_lib.hp_mesh2d_factors(mesh, out.ctypes.data), "hp_mesh2d_factors")
    return out


def hp_mesh2d_sync(mesh, stream=None):
    _check(_lib.hp_mesh2d_sync(mesh, _stream(stream)), "hp_mesh2d_sync")


def hp_mesh2d_destroy(mesh):
    _lib.hp_mesh2d_destroy(mesh)


def hp_mesh_layout(mesh, n_elem):
    co = np.zeros(n_elem + 1, dtype=np.int64)
    po = np.zeros(n_elem + 1, dtype=np.int64)
    nc, nph = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.hp_mesh_layout(mesh, co.ctypes.data, po.ctypes.data, ctypes.byref(nc), ctypes.byref(nph)),
           "hp_mesh_layout")
    return co, po, nc.value, nph.value


def hp_geom_factors(mesh, stream=None):
    _check(_lib.hp_geom_factors(mesh, _stream(stream)), "hp_geom_factors")


def hp_geom_copy(mesh, n_phys, want_deriv=False):
    out7 = np.zeros(7 * n_phys)
    out9 = np.zeros(9 * n_phys) if want_deriv else None
    _check(_lib.hp_geom_copy(mesh, out7.ctypes.data, None if out9 is None else out9.ctypes.data), "hp_geom_copy")
    return out7, out9


def hp_op_create(mesh, kind, strategy=HP_STRAT_SUMFAC, dtype=HP_FP64):
    h = _vp()
    _check(_lib.hp_op_create(mesh, int(kind), int(strategy), int(dtype), ctypes.byref(h)), "hp_op_create")
    return h.value


def hp_op_apply(op, lam, x, y, stream=None):
    _check(_lib.hp_op_apply(op, float(lam), _ptr(x), _ptr(y), _stream(stream)), "hp_op_apply")


def hp_op_apply_graph(op, lam, x, y, stream=None):
    _check(_lib.hp_op_apply_graph(op, float(lam), _ptr(x), _ptr(y), _stream(stream)), "hp_op_apply_graph")


def hp_op_tune(op, lam, x, y, stream=None):
    _check(_lib.hp_op_tune(op, float(lam), _ptr(x), _ptr(y), _stream(stream)), "hp_op_tune")


def hp_op_tiles(op, n_blocks, tiles=None):
    """Return the per-block tile variants, or set them when ``tiles`` is given."""
    arr = np.zeros(n_blocks, dtype=np.int32) if tiles is None else np.ascontiguousarray(tiles, dtype=np.int32)
    _check(_lib.hp_op_tiles(op, arr.ctypes.data, int(n_blocks), 0 if tiles is None else 1), "hp_op_tiles")
    return arr


def hp_op_set_advection(op, velocity):
    """Constant advection velocity (3 floats) of an HP_ADVECTION_DIFFUSION_REACTION op."""
    v = np.ascontiguousarray(velocity, dtype=np.float64)
    if v.shape != (3,):
        raise ValueError("velocity must have 3 components")
    _check(_lib.hp_op_set_advection(op, v.ctypes.data), "hp_op_set_advection")


def hp_op_set_batching(op, mode):
    """0: one kernel per block (graph of concurrent nodes); 1: one persistent work-list launch."""
    _check(_lib.hp_op_set_batching(op, int(mode)), "hp_op_set_batching")


def hp_op_set_deterministic(op, deterministic):
    """Fixed-order (True) or atomic (False, the default) sum of the tensor-core
    operators' split tiles."""
    _check(_lib.hp_op_set_deterministic(op, 1 if deterministic else 0), "hp_op_set_deterministic")


def hp_op_set_collocated(op, collocated):
    """Collocated (True, the default) or non-collocated (False, FP64 only) form of
    the op's sum-factorised Laplacian / Helmholtz blocks."""
    _check(_lib.hp_op_set_collocated(op, 1 if collocated else 0), "hp_op_set_collocated")


def hp_op_sync(op, stream=None):
    _check(_lib.hp_op_sync(op, _stream(stream)), "hp_op_sync")


def hp_op_work(op):
    d, f, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.hp_op_work(op, ctypes.byref(d), ctypes.byref(f), ctypes.byref(b)), "hp_op_work")
    return d.value, f.value, b.value


def hp_op_block_work(op, block):
    """(n_elem, output DOFs, collocated flops, executed flops, bytes) of one
    block (-1: the whole operator)."""
    n = ctypes.c_int64(0)
    d = ctypes.c_int64(0)
    f = ctypes.c_double(0)
    fx = ctypes.c_double(0)
    b = ctypes.c_double(0)
    _check(_lib.hp_op_block_work(op, int(block), ctypes.byref(n), ctypes.byref(d), ctypes.byref(f), ctypes.byref(fx),
                                 ctypes.byref(b)), "hp_op_block_work")
    return n.value, d.value, f.value, fx.value, b.value


def hp_op_apply_block(op, block, lam, x, y, stream=None):
    _check(_lib.hp_op_apply_block(op, int(block), float(lam), _ptr(x), _ptr(y), _stream(stream)), "hp_op_apply_block")


def hp_peak_fp64(device=0, iters=20000, stream=None):
    """(TFLOP/s, ms) of the library's FP64 FMA-loop kernel on `device`."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.hp_peak_fp64(int(device), int(iters), ctypes.byref(t), ctypes.byref(ms), _stream(stream)),
           "hp_peak_fp64")
    return t.value, ms.value


def hp_op_destroy(op):
    _lib.hp_op_destroy(op)


def hp_mesh_destroy(mesh):
    _lib.hp_mesh_destroy(mesh)


def hp_status_str(s):
    return _lib.hp_status_str(int(s)).decode()


def hp_last_error():
    return _lib.hp_last_error().decode()


def hp_op_strategies(op, n_blocks, strategies=None):
    """Return the per-block strategies, or set them when ``strategies`` is given."""
    arr = np.zeros(n_blocks, dtype=np.int32) if strategies is None else np.ascontiguousarray(strategies, np.int32)
    _check(_lib.hp_op_strategies(op, arr.ctypes.data, int(n_blocks), 0 if strategies is None else 1),
           "hp_op_strategies")
    return arr


def hp_op_block_features(op, n_blocks):
    f = np.zeros((n_blocks, 5), dtype=np.float32)
    _check(_lib.hp_op_block_features(op, f.ctypes.data, int(n_blocks)), "hp_op_block_features")
    return f


def hp_op_schedule(op, mlp, stream=None):
    _check(_lib.hp_op_schedule(op, mlp, _stream(stream)), "hp_op_schedule")


def hp_op_schedule_mlp(op, mlp, graph_launch=0, stream=None):
    _check(_lib.hp_op_schedule_mlp(op, mlp, int(graph_launch), _stream(stream)), "hp_op_schedule_mlp")


def hp_op_schedule_exhaustive(op, lam, x, y, n_blocks, stream=None):
    """Per-block times [n_blocks, 4] (ms; columns SUMFAC, ELEMAT, HYBRID, MATRIX;
    1e30 where not built) after choosing the fastest per block."""
    t = np.zeros((n_blocks, 4), dtype=np.float32)
    _check(_lib.hp_op_schedule_exhaustive(op, float(lam), _ptr(x), _ptr(y), t.ctypes.data, _stream(stream)),
           "hp_op_schedule_exhaustive")
    return t


def hp_op_schedule_graph(op, lam, x, y, reps=5, passes=1, stream=None):
    """Coordinate descent on the concurrent graph's time; returns its final median ms."""
    t = ctypes.c_float(0.0)
    _check(_lib.hp_op_schedule_graph(op, float(lam), _ptr(x), _ptr(y), int(reps), int(passes), ctypes.byref(t),
                                     _stream(stream)), "hp_op_schedule_graph")
    return t.value


def hp_mlp_create(n_in, n_hidden, n_out, seed=0, device=0):
    h = _vp()
    _check(_lib.hp_mlp_create(int(n_in), int(n_hidden), int(n_out), int(seed), int(device), ctypes.byref(h)),
           "hp_mlp_create")
    return h.value


def hp_mlp_info(mlp):
    a, b, c, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(_lib.hp_mlp_info(mlp, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)), "hp_mlp_info")
    return a.value, b.value, c.value, d.value


def hp_mlp_params(mlp, params=None):
    """Return the flat FP32 parameters, or set them when ``params`` is given."""
    n = hp_mlp_info(mlp)[3]
    arr = np.zeros(n, dtype=np.float32) if params is None else np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib.hp_mlp_params(mlp, arr.ctypes.data, int(n), 0 if params is None else 1), "hp_mlp_params")
    return arr


def hp_mlp_forward(mlp, x, batch, y, stream=None):
    _check(_lib.hp_mlp_forward(mlp, _ptr(x), int(batch), _ptr(y), _stream(stream)), "hp_mlp_forward")


def hp_mlp_grad(mlp, x, t, batch, grad, loss=None, stream=None):
    _check(_lib.hp_mlp_grad(mlp, _ptr(x), _ptr(t), int(batch), _ptr(grad), _ptr(loss), _stream(stream)),
           "hp_mlp_grad")


def hp_mlp_adam_step(mlp, x, t, batch, lr, loss=None, stream=None):
    _check(_lib.hp_mlp_adam_step(mlp, _ptr(x), _ptr(t), int(batch), float(lr), _ptr(loss), _stream(stream)),
           "hp_mlp_adam_step")


def hp_mlp_destroy(mlp):
    _lib.hp_mlp_destroy(mlp)


def hp_mlp_grad_noalloc(params, n_in, n_hidden, n_out, x, t, batch, grad, loss=None, stream=None):
    """Gradient with caller-passed parameters and no device allocation (fixed 2^20-float scratch)."""
    _check(_lib.hp_mlp_grad_noalloc(_ptr(params), int(n_in), int(n_hidden), int(n_out), _ptr(x), _ptr(t),
                                    int(batch), _ptr(grad), _ptr(loss), _stream(stream)), "hp_mlp_grad_noalloc")


class hp_solve_opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("mixed", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("inner_max_iter", ctypes.c_int), ("max_refinements", ctypes.c_int),
                ("schedule", ctypes.c_int)]


class hp_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("inner_iterations", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double)]


_lib.hp_mesh_points.argtypes = [_vp, _vp, _vp]
_lib.hp_c0_create.argtypes = [_vp, ctypes.POINTER(_vp)]
_lib.hp_c0_info.argtypes = [_vp, _vp, _vp]
_lib.hp_c0_map_host.argtypes = [ctypes.POINTER(hp_mesh_desc), _vp, _vp, _vp, _vp]
_lib.hp_c0_maps.argtypes = [_vp, _vp, _vp, _vp]
_lib.hp_c0_gather.argtypes = [_vp, _vp, _vp, _vp]
_lib.hp_c0_assemble.argtypes = [_vp, _vp, _vp, ctypes.c_int, _vp]
_lib.hp_solve.argtypes = [_vp, ctypes.c_double, _vp, _vp, ctypes.POINTER(hp_solve_opts),
                          ctypes.POINTER(hp_solve_stats), _vp]
_lib.hp_c0_destroy.argtypes = [_vp]
_lib.hp_c0_diagonal.argtypes = [_vp, ctypes.c_double, _vp, ctypes.c_int, _vp]
_lib.hp_c0_diagonal.restype = ctypes.c_int
for _f in ("hp_mesh_points", "hp_c0_create", "hp_c0_info", "hp_c0_map_host", "hp_c0_maps", "hp_c0_gather",
           "hp_c0_assemble", "hp_solve"):
    getattr(_lib, _f).restype = ctypes.c_int


def _desc(mesh):
    keep = dict(shape=np.ascontiguousarray(mesh["shape"], dtype=np.uint8),
                P=np.ascontiguousarray(mesh["P"], dtype=np.uint8),
                Q=np.ascontiguousarray(mesh["Q"], dtype=np.uint8),
                vert=np.ascontiguousarray(mesh["vert"], dtype=np.int64),
                xyz=np.ascontiguousarray(mesh["xyz"], dtype=np.float64),
                curved=np.ascontiguousarray(mesh["curved"], dtype=np.uint8))
    d = hp_mesh_desc(int(mesh["n_elem"]), keep["shape"].ctypes.data, keep["P"].ctypes.data,
                     keep["Q"].ctypes.data, keep["vert"].ctypes.data, keep["xyz"].ctypes.data,
                     int(keep["xyz"].shape[0]), keep["curved"].ctypes.data, int(mesh["deformation"]),
                     int(mesh.get("geometry", 0)))
    return d, keep


def hp_mesh_points(mesh, xyz, stream=None):
    _check(_lib.hp_mesh_points(mesh, _ptr(xyz), _stream(stream)), "hp_mesh_points")


def hp_c0_map_host(mesh, n_coeff):
    """Host-side C0 numbering: (gid, sign, boundary, n_global)."""
    d, keep = _desc(mesh)
    gid = np.zeros(n_coeff, dtype=np.int64)
    sign = np.zeros(n_coeff, dtype=np.int8)
    bnd = np.zeros(n_coeff, dtype=np.uint8)
    ng = ctypes.c_int64()
    _check(_lib.hp_c0_map_host(ctypes.byref(d), gid.ctypes.data, sign.ctypes.data, bnd.ctypes.data,
                               ctypes.byref(ng)), "hp_c0_map_host")
    return gid, sign, bnd[:ng.value].copy(), ng.value


def hp_c0_create(mesh):
    h = _vp()
    _check(_lib.hp_c0_create(mesh, ctypes.byref(h)), "hp_c0_create")
    return h.value


def hp_c0_info(c0):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.hp_c0_info(c0, ctypes.byref(a), ctypes.byref(b)), "hp_c0_info")
    return a.value, b.value


def hp_c0_maps(c0, n_coeff):
    ng = hp_c0_info(c0)[0]
    gid = np.zeros(n_coeff, dtype=np.int64)
    sign = np.zeros(n_coeff, dtype=np.int8)
    bnd = np.zeros(ng, dtype=np.uint8)
    _check(_lib.hp_c0_maps(c0, gid.ctypes.data, sign.ctypes.data, bnd.ctypes.data), "hp_c0_maps")
    return gid, sign, bnd


def hp_c0_gather(c0, glob, loc, stream=None):
    _check(_lib.hp_c0_gather(c0, _ptr(glob), _ptr(loc), _stream(stream)), "hp_c0_gather")


def hp_c0_assemble(c0, loc, glob, mask_boundary=True, stream=None):
    _check(_lib.hp_c0_assemble(c0, _ptr(loc), _ptr(glob), 1 if mask_boundary else 0, _stream(stream)),
           "hp_c0_assemble")


def hp_solve(c0, lam, rhs, x, tol=1e-10, max_iter=20000, mixed=False, inner_tol=1e-5, inner_max_iter=20000,
             max_refinements=20, schedule=False, stream=None):
    """Returns (status, stats); raises for errors other than HP_ERR_NOT_CONVERGED.
    mixed: 0 / False FP64 PCG, 1 / True FP32 inner PCG with FP64 refinement,
    2 / 3 the same with the TF32 / BF16 tensor-core inner operator.
    schedule: choose the operators' per-block strategies by the graph-aware
    schedule (stored matrices included) before the first solve."""
    o = hp_solve_opts(float(tol), int(max_iter), int(mixed), float(inner_tol), int(inner_max_iter),
                      int(max_refinements), 1 if schedule else 0)
    st = hp_solve_stats()
    rc = _lib.hp_solve(c0, float(lam), _ptr(rhs), _ptr(x), ctypes.byref(o), ctypes.byref(st), _stream(stream))
    if rc not in (HP_OK, HP_ERR_NOT_CONVERGED):
        raise HpError(rc, "hp_solve")
    return rc, dict(iterations=st.iterations, inner_iterations=st.inner_iterations, refinements=st.refinements,
                    rel_residual=st.rel_residual)


def hp_c0_destroy(c0):
    _lib.hp_c0_destroy(c0)


def hp_c0_diagonal(c0, lam, diag, local=False, stream=None):
    _check(_lib.hp_c0_diagonal(c0, float(lam), _ptr(diag), 1 if local else 0, _stream(stream)), "hp_c0_diagonal")


# ---------------------------------------------------------------- multi-GPU layout (host only)
_lib.hp_partition.argtypes = [ctypes.POINTER(hp_mesh_desc), _vp, ctypes.c_int, ctypes.c_int, _vp]
_lib.hp_halo_create.argtypes = [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int64, _vp, ctypes.c_int, ctypes.c_int,
                                ctypes.POINTER(_vp)]
_lib.hp_halo_info.argtypes = [_vp, _i64p, _i64p, _i64p]
_lib.hp_halo_counts.argtypes = [_vp, _vp, _vp, _vp, _vp]
_lib.hp_halo_maps.argtypes = [_vp, _vp, _vp, _vp]
_lib.hp_halo_gather.argtypes = [_vp, _vp, _vp]
_lib.hp_halo_reduce_pack.argtypes = [_vp, _vp, _vp]
_lib.hp_halo_reduce_sum.argtypes = [_vp, _vp, _vp, _vp]
_lib.hp_halo_bcast_pack.argtypes = [_vp, _vp, _vp]
_lib.hp_halo_bcast_unpack.argtypes = [_vp, _vp, _vp, _vp]
_lib.hp_halo_destroy.argtypes = [_vp]
_lib.hp_xdot_acc.argtypes = [_vp, _vp, ctypes.c_int64, _vp]
_lib.hp_xacc_round.argtypes = [_vp, _dp]
for _f in ("hp_partition", "hp_halo_create", "hp_halo_info", "hp_halo_counts", "hp_halo_maps", "hp_halo_gather",
           "hp_halo_reduce_pack", "hp_halo_reduce_sum", "hp_halo_bcast_pack", "hp_halo_bcast_unpack", "hp_xdot_acc",
           "hp_xacc_round", "hp_xacc_limbs"):
    getattr(_lib, _f).restype = ctypes.c_int
HP_XACC_LIMBS = _lib.hp_xacc_limbs()


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def hp_partition(mesh, nparts, method=0, cost=None):
    """Element partition (int32 part ids) balanced by cost (default: the
    collocated Helmholtz flops of each element); method 0: ranges of the
    block order, 1: recursive coordinate bisection."""
    d, keep = _desc(mesh)
    part = np.zeros(int(mesh["n_elem"]), dtype=np.int32)
    c = None if cost is None else _f64(cost)
    _check(_lib.hp_partition(ctypes.byref(d), None if c is None else c.ctypes.data, int(nparts), int(method),
                             part.ctypes.data), "hp_partition")
    return part


class Halo:
    """One rank's halo plan (hp_halo_*): sizes, per-peer message counts, maps
    and the host pack / sum / unpack steps on numpy float64 arrays."""

    def __init__(self, gid, sign, coeff_offset, n_global, part, nparts, rank):
        gid = np.ascontiguousarray(gid, dtype=np.int64)
        sign = np.ascontiguousarray(sign, dtype=np.int8)
        co = np.ascontiguousarray(coeff_offset, dtype=np.int64)
        part = np.ascontiguousarray(part, dtype=np.int32)
        h = _vp()
        _check(_lib.hp_halo_create(gid.ctypes.data, sign.ctypes.data, co.ctypes.data, len(co) - 1, int(n_global),
                                   part.ctypes.data, int(nparts), int(rank), ctypes.byref(h)), "hp_halo_create")
        self.h, self.nparts, self.rank = h.value, int(nparts), int(rank)
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(_lib.hp_halo_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "hp_halo_info")
        self.n_local, self.n_touched, self.n_owned = a.value, b.value, c.value
        self.counts = [np.zeros(self.nparts, dtype=np.int64) for _ in range(4)]
        _check(_lib.hp_halo_counts(self.h, *[x.ctypes.data for x in self.counts]), "hp_halo_counts")
        self.reduce_send, self.reduce_recv, self.bcast_send, self.bcast_recv = self.counts
        self.local_index = np.zeros(self.n_local, dtype=np.int64)
        self.touched_gid = np.zeros(self.n_touched, dtype=np.int64)
        self.owned_gid = np.zeros(self.n_owned, dtype=np.int64)
        _check(_lib.hp_halo_maps(self.h, self.local_index.ctypes.data, self.touched_gid.ctypes.data,
                                 self.owned_gid.ctypes.data), "hp_halo_maps")

    def gather(self, touched):
        touched = _f64(touched)
        out = np.zeros(self.n_local)
        _check(_lib.hp_halo_gather(self.h, touched.ctypes.data, out.ctypes.data), "hp_halo_gather")
        return out

    def reduce_pack(self, local):
        local = _f64(local)
        out = np.zeros(int(self.reduce_send.sum()))
        _check(_lib.hp_halo_reduce_pack(self.h, local.ctypes.data, out.ctypes.data), "hp_halo_reduce_pack")
        return out

    def reduce_sum(self, local, recv):
        local, recv = _f64(local), _f64(recv)
        out = np.zeros(self.n_owned)
        _check(_lib.hp_halo_reduce_sum(self.h, local.ctypes.data, recv.ctypes.data, out.ctypes.data),
               "hp_halo_reduce_sum")
        return out

    def bcast_pack(self, owned):
        owned = _f64(owned)
        out = np.zeros(int(self.bcast_send.sum()))
        _check(_lib.hp_halo_bcast_pack(self.h, owned.ctypes.data, out.ctypes.data), "hp_halo_bcast_pack")
        return out

    def bcast_unpack(self, owned, recv):
        owned, recv = _f64(owned), _f64(recv)
        out = np.zeros(self.n_touched)
        _check(_lib.hp_halo_bcast_unpack(self.h, owned.ctypes.data, recv.ctypes.data, out.ctypes.data),
               "hp_halo_bcast_unpack")
        return out

    def __del__(self):
        if getattr(self, "h", None):
            _lib.hp_halo_destroy(self.h)
            self.h = None


def hp_xdot_acc(x, y, acc=None):
    """Add sum x_i y_i exactly into an int64 accumulator (new if None); returns it."""
    x, y = _f64(x), _f64(y)
    if acc is None:
        acc = np.zeros(HP_XACC_LIMBS, dtype=np.int64)
    _check(_lib.hp_xdot_acc(x.ctypes.data, y.ctypes.data, len(x), acc.ctypes.data), "hp_xdot_acc")
    return acc


def hp_xacc_round(acc):
    acc = np.ascontiguousarray(acc, dtype=np.int64)
    out = ctypes.c_double()
    _check(_lib.hp_xacc_round(acc.ctypes.data, ctypes.byref(out)), "hp_xacc_round")
    return out.value


def hp_xacc_limbs():
    return HP_XACC_LIMBS


def hp_halo_create(gid, sign, coeff_offset, n_global, part, nparts, rank):
    return Halo(gid, sign, coeff_offset, n_global, part, nparts, rank)


def hp_halo_info(halo):
    return halo.n_local, halo.n_touched, halo.n_owned


def hp_halo_counts(halo):
    return halo.reduce_send, halo.reduce_recv, halo.bcast_send, halo.bcast_recv


def hp_halo_maps(halo):
    return halo.local_index, halo.touched_gid, halo.owned_gid


def hp_halo_gather(halo, touched):
    return halo.gather(touched)


def hp_halo_reduce_pack(halo, local):
    return halo.reduce_pack(local)


def hp_halo_reduce_sum(halo, local, recv):
    return halo.reduce_sum(local, recv)


def hp_halo_bcast_pack(halo, owned):
    return halo.bcast_pack(owned)


def hp_halo_bcast_unpack(halo, owned, recv):
    return halo.bcast_unpack(owned, recv)


def hp_halo_destroy(halo):
    halo.__del__()
