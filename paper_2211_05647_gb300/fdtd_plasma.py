"""Thin ctypes binding of the C ABI in ``include/fdtd_plasma.h``.

The functions keep the C names (``fdtd_plasma_create`` ...) and only marshal
arguments; every step of the computation runs in the CUDA library.  PyTorch
supplies device memory (through the allocator callback) and the stream.  If
the library has not been built the import fails loudly: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libfdtd_plasma.so")

# ---------------------------------------------------------------- constants
FDTD_OK, FDTD_ERR_INVAL, FDTD_ERR_NOMEM, FDTD_ERR_CUDA = 0, -1, -2, -3
FDTD_ERR_UNSTABLE, FDTD_ERR_NONFINITE, FDTD_ERR_TIMEOUT, FDTD_ERR_STATE = -4, -5, -6, -7
STATUS = {0: "OK", -1: "INVAL", -2: "NOMEM", -3: "CUDA", -4: "UNSTABLE", -5: "NONFINITE", -6: "TIMEOUT", -7: "STATE"}
PRECISION = {"f32": 0, "f64": 1}
DF_DTYPE = {"f32": 0, "bf16": 1, "f64": 2}
VGRID = {"signed1d": 0, "cart2d": 1, "speed3d": 2}
NU_MODEL = {"nsv": 0, "const": 1, "table": 2}
F0_MODEL = {"maxwell": 0, "druyvesteyn": 1}
SRC_KIND = {"none": 0, "gauss_sine": 1, "gauss": 2}
SRC_LOC = {"point": 0, "sheet": 1}
QUANTITY = {"ex": 0, "ey": 1, "ez": 2, "hx": 3, "hy": 4, "hz": 5, "j": 6, "df": 7, "f0": 8}


class FdtdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fdtd_plasma error {STATUS.get(code, code)}: {msg}")
        self.code = code


# ---------------------------------------------------------------- structs
class fdtd_grid_desc(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("dx", ctypes.c_double), ("courant", ctypes.c_double),
                ("cpml_cells", ctypes.c_int32), ("mur", ctypes.c_int32),
                ("cpml_order", ctypes.c_double), ("cpml_sigma_factor", ctypes.c_double),
                ("cpml_kappa_max", ctypes.c_double), ("cpml_alpha_min", ctypes.c_double),
                ("cpml_alpha_max", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class fdtd_runtime_desc(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", ctypes.c_void_p)]


class fdtd_source_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("location", ctypes.c_int32),
                ("amp", ctypes.c_double), ("fc", ctypes.c_double), ("tau", ctypes.c_double), ("t0", ctypes.c_double),
                ("i", ctypes.c_int64), ("j", ctypes.c_int64), ("k", ctypes.c_int64),
                ("i0", ctypes.c_int64), ("i1", ctypes.c_int64), ("j0", ctypes.c_int64), ("j1", ctypes.c_int64)]


class fdtd_plasma_desc(ctypes.Structure):
    _fields_ = [("density", ctypes.c_void_p), ("density_on_device", ctypes.c_int32),
                ("vgrid", ctypes.c_int32), ("nv", ctypes.c_int32), ("nv_perp", ctypes.c_int32),
                ("te_ev", ctypes.c_double), ("vmax_vth", ctypes.c_double), ("nu0", ctypes.c_double),
                ("nu_model", ctypes.c_int32), ("f_dtype", ctypes.c_int32), ("nonlinear", ctypes.c_int32),
                ("f0_model", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("s_speed", ctypes.c_void_p), ("s_sigma", ctypes.c_void_p), ("s_n", ctypes.c_int64),
                ("evolve_f0", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mass_ratio", ctypes.c_double), ("tg_ev", ctypes.c_double)]


class fdtd_diag(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("energy_plain", ctypes.c_double), ("number", ctypes.c_double),
                ("number_max_cell", ctypes.c_double), ("number_abs", ctypes.c_double),
                ("finite", ctypes.c_int64), ("step", ctypes.c_int64)]


class fdtd_diag_arrays(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("nz", ctypes.c_int64),
                ("dx", ctypes.c_double), ("courant", ctypes.c_double),
                ("fields", ctypes.c_void_p * 6), ("df", ctypes.c_void_p),
                ("f_dtype", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("nslots", ctypes.c_int64), ("nnode", ctypes.c_int64), ("dV", ctypes.c_void_p)]


class fdtd_tune_result(ctypes.Structure):
    _fields_ = [("kin_vpl", ctypes.c_int32), ("kin_l", ctypes.c_int32), ("kin_blocks_per_sm", ctypes.c_int32),
                ("block_x", ctypes.c_int32), ("block_y", ctypes.c_int32), ("block_z", ctypes.c_int32),
                ("kin_ms", ctypes.c_double), ("stencil_ms", ctypes.c_double),
                ("cells_per_thread", ctypes.c_int32), ("stencil_tz", ctypes.c_int32),
                ("kin_stages", ctypes.c_int32), ("fused_rows", ctypes.c_int32)]


class fdtd_closure_desc(ctypes.Structure):
    _fields_ = [("params", ctypes.c_void_p), ("params_on_device", ctypes.c_int32), ("engine", ctypes.c_int32),
                ("e_scale", ctypes.c_double), ("j_scale", ctypes.c_double), ("n_scale", ctypes.c_double),
                ("rho", ctypes.c_double), ("n_train_max", ctypes.c_double), ("beta", ctypes.c_double)]


class fdtd_subdomain_desc(ctypes.Structure):
    _fields_ = [("axis", ctypes.c_int32), ("reserved", ctypes.c_int32), ("n_global", ctypes.c_int64),
                ("offset", ctypes.c_int64), ("extent", ctypes.c_int64)]


HALO = {"e": 0, "h": 1}


class fdtd_closure_scales_t(ctypes.Structure):
    _fields_ = [("e_scale", ctypes.c_double), ("j_scale", ctypes.c_double), ("n_scale", ctypes.c_double),
                ("rho", ctypes.c_double), ("beta", ctypes.c_double)]


MLP_NPARAMS = 18945
MLP_NIN = 17
MLP_NHID = 128


class fdtd_run_desc(ctypes.Structure):
    _fields_ = [("grid", fdtd_grid_desc), ("plasma", fdtd_plasma_desc), ("source", fdtd_source_desc)]


# ---------------------------------------------------------------- library
_lib = None
_lib_lock = threading.Lock()

# name -> (restype, argtypes); every symbol the header declares
SIGNATURES = {
    "fdtd_plasma_create": (ctypes.c_int, [ctypes.POINTER(fdtd_grid_desc), ctypes.POINTER(fdtd_runtime_desc),
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "fdtd_plasma_set_source": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fdtd_source_desc)]),
    "fdtd_plasma_set_plasma": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fdtd_plasma_desc)]),
    "fdtd_plasma_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "fdtd_plasma_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "fdtd_plasma_time_kernels": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)]),
    "fdtd_plasma_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fdtd_tune_result)]),
    "fdtd_plasma_read_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                               ctypes.c_int]),
    "fdtd_plasma_write_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                                ctypes.c_int]),
    "fdtd_plasma_quantity_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    "fdtd_plasma_plasma_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                                ctypes.POINTER(ctypes.c_int64)]),
    "fdtd_plasma_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int64)]),
    "fdtd_plasma_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fdtd_diag)]),
    "fdtd_plasma_poynting": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_double)]),
    "fdtd_plasma_check_canaries": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)]),
    "fdtd_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]),
    "fdtd_selftest_timed_wait": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32)]),
    "fdtd_plasma_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]),
    "fdtd_plasma_launch_shapes": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fdtd_tune_result)]),
    "fdtd_plasma_set_ports": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                             ctypes.POINTER(ctypes.c_int64), ctypes.c_int32,
                                             ctypes.POINTER(ctypes.c_double)]),
    "fdtd_plasma_read_ports": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t]),
    "fdtd_plasma_state_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "fdtd_plasma_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]),
    "fdtd_plasma_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]),
    "fdtd_plasma_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fdtd_plasma_set_closure": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fdtd_closure_desc)]),
    "fdtd_plasma_closure_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                                 ctypes.POINTER(ctypes.c_int64)]),
    "fdtd_plasma_set_recording": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                 ctypes.c_double, ctypes.c_uint64]),
    "fdtd_mlp_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "fdtd_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_void_p]),
    "fdtd_mlp_forward_tc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
    "fdtd_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                          ctypes.c_void_p]),
    "fdtd_mlp_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_void_p]),
    "fdtd_closure_workspace_bytes": (ctypes.c_size_t, []),
    "fdtd_closure_scales": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, ctypes.POINTER(fdtd_closure_scales_t),
                                           ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "fdtd_closure_dataset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(fdtd_closure_scales_t),
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fdtd_mlp_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "fdtd_mlp_gather": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "fdtd_mlp_train_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "fdtd_mlp_train_epoch": (ctypes.c_int, [ctypes.c_void_p] * 6 + [ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                                                                   ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                                                   ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                                                   ctypes.c_size_t, ctypes.c_void_p]),
    "fdtd_batch_create": (ctypes.c_int, [ctypes.POINTER(fdtd_run_desc), ctypes.c_int32,
                                         ctypes.POINTER(fdtd_runtime_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "fdtd_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "fdtd_batch_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.c_int]),
    "fdtd_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_double)]),
    "fdtd_batch_write": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_int]),
    "fdtd_batch_quantity_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int]),
    "fdtd_batch_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "fdtd_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fdtd_batch_destroy": (None, [ctypes.c_void_p]),
    "fdtd_diagnostics_noalloc": (ctypes.c_int, [ctypes.POINTER(fdtd_diag_arrays), ctypes.POINTER(ctypes.c_double),
                                                ctypes.c_int, ctypes.c_void_p]),
    "fdtd_plasma_create_subdomain": (ctypes.c_int, [ctypes.POINTER(fdtd_grid_desc), ctypes.POINTER(fdtd_subdomain_desc),
                                                    ctypes.POINTER(fdtd_runtime_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "fdtd_plasma_step_half": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fdtd_plasma_halo_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    "fdtd_plasma_halo_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "fdtd_plasma_halo_unpack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "fdtd_plasma_destroy": (None, [ctypes.c_void_p]),
}


def load_library(path: str = LIB_PATH):
    """Load the CUDA library; raises if it is missing (no fallback)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(lib, h, rc):
    if rc != FDTD_OK:
        msg = lib.fdtd_plasma_last_error(h)
        raise FdtdError(rc, msg.decode() if msg else "")


# ---------------------------------------------------------- torch plumbing
class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, handed to the C side
    through the fdtd_runtime_desc callbacks."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            t = self.torch.empty(int(nbytes) + 256, dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        p = t.data_ptr()
        p_al = (p + 255) & ~255
        self.live[p_al] = t
        return p_al

    def _free(self, ptr, ctx):
        self.live.pop(ptr, None)


def _grid_desc(grid: dict) -> fdtd_grid_desc:
    g = fdtd_grid_desc()
    g.ndim = int(grid["ndim"])
    g.precision = PRECISION[grid.get("precision", "f32")]
    g.nx, g.ny, g.nz = int(grid.get("nx", 1)), int(grid.get("ny", 1)), int(grid.get("nz", 1))
    g.dx, g.courant = float(grid["dx"]), float(grid.get("courant", 0.5))
    g.cpml_cells, g.mur = int(grid.get("cpml_cells", 0)), int(grid.get("mur", 0))
    g.cpml_order = float(grid.get("cpml_order", 3.0))
    g.cpml_sigma_factor = float(grid.get("cpml_sigma_factor", 1.3))
    g.cpml_kappa_max = float(grid.get("cpml_kappa_max", 7.0))
    g.cpml_alpha_min = float(grid.get("cpml_alpha_min", 0.0))
    g.cpml_alpha_max = float(grid.get("cpml_alpha_max", 0.05))
    return g


def _source_desc(kind="gauss_sine", location="point", amp=1.0, fc=0.0, tau=1.0, t0=0.0, i=0, j=0, k=0, i0=0, i1=0,
                 j0=0, j1=0) -> fdtd_source_desc:
    return fdtd_source_desc(SRC_KIND[kind], SRC_LOC[location], amp, fc, tau, t0, i, j, k, i0, i1, j0, j1)


def _plasma_desc(density_ptr, on_device, vgrid="signed1d", nv=64, nv_perp=1, te_ev=1.0, vmax_vth=6.0, nu0=0.0,
                 nu_model="nsv", f_dtype="f32", nonlinear=0, seed=0, f0_model="maxwell", s_table=None,
                 evolve_f0=0, mass_ratio=0.0, tg_ev=0.0):
    """Returns (descriptor, arrays the descriptor points into: keep them alive
    until the create / set_plasma call has returned)."""
    d = fdtd_plasma_desc()
    d.density, d.density_on_device = density_ptr, on_device
    d.vgrid, d.nv, d.nv_perp = VGRID[vgrid], int(nv), int(nv_perp)
    d.te_ev, d.vmax_vth, d.nu0 = float(te_ev), float(vmax_vth), float(nu0)
    d.nu_model, d.f_dtype, d.nonlinear = NU_MODEL[nu_model], DF_DTYPE[f_dtype], int(nonlinear)
    d.f0_model = F0_MODEL[f0_model]
    d.evolve_f0, d.mass_ratio, d.tg_ev = int(evolve_f0), float(mass_ratio), float(tg_ev)
    d.seed = int(seed)
    keep = ()
    if s_table is not None:
        sp = np.ascontiguousarray(s_table[0], dtype=np.float64)
        sg = np.ascontiguousarray(s_table[1], dtype=np.float64)
        if sp.shape != sg.shape or sp.ndim != 1:
            raise ValueError("s_table: (speeds, cross-sections), two 1-D arrays of equal length")
        d.s_speed, d.s_sigma, d.s_n = sp.ctypes.data, sg.ctypes.data, sp.size
        keep = (sp, sg)
    return d, keep


# ------------------------------------------------------------ closure network
def selftest_wait_timeout(max_iter: int = 1000) -> bool:
    """Run the bounded-wait self-test; True when the wait gave up as designed."""
    lib = load_library()
    out = ctypes.c_int32(-1)
    _check(lib, None, lib.fdtd_selftest_wait_timeout(int(max_iter), ctypes.byref(out)))
    return out.value == 1


def selftest_timed_wait(limit_us: int = 2000) -> bool:
    """Run the wall-clock-bounded wait self-test; True when the wait gave up as designed."""
    lib = load_library()
    out = ctypes.c_int32(-1)
    _check(lib, None, lib.fdtd_selftest_timed_wait(int(limit_us), ctypes.byref(out)))
    return out.value == 1


def mlp_forward(params, x, stream=None):
    """y = MLP(x) on the GPU (params [18945], x [B, 17]; torch float32 cuda tensors)."""
    import torch
    lib = load_library()
    x = x.contiguous()
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    st = (stream or torch.cuda.current_stream(x.device)).cuda_stream
    _check(lib, None, lib.fdtd_mlp_forward(params.data_ptr(), x.data_ptr(), x.shape[0], y.data_ptr(), st))
    return y


def mlp_forward_tc(params, x, stream=None):
    """tcgen05 forward; returns (y, err) with err the device flag of a bounded wait that gave up."""
    import torch
    lib = load_library()
    x = x.contiguous()
    y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
    err = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = (stream or torch.cuda.current_stream(x.device)).cuda_stream
    _check(lib, None, lib.fdtd_mlp_forward_tc(params.data_ptr(), x.data_ptr(), x.shape[0], y.data_ptr(),
                                              err.data_ptr(), st))
    return y, err


class MlpTrainer:
    """Mean-squared-error training of the closure network with the library's
    own GPU kernels: loss + gradient (fdtd_mlp_loss_grad) and Adam
    (fdtd_mlp_adam), on torch device buffers."""

    def __init__(self, params, batch: int, lr=1e-3, betas=(0.9, 0.999), eps=1e-8):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.p = params
        self.dev = params.device
        self.grad = torch.zeros_like(params)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.ws_bytes = self.lib.fdtd_mlp_workspace_bytes(batch)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.dev)
        self.batch = batch
        self.t = 0
        self.lr, self.betas, self.eps = lr, betas, eps

    def loss_grad(self, x, t):
        st = self.torch.cuda.current_stream(self.dev).cuda_stream
        assert x.shape[0] <= self.batch
        _check(self.lib, None, self.lib.fdtd_mlp_loss_grad(self.p.data_ptr(), x.data_ptr(), t.data_ptr(), x.shape[0],
                                                           self.grad.data_ptr(), self.loss.data_ptr(),
                                                           self.ws.data_ptr(), self.ws_bytes, st))
        return self.loss, self.grad

    def epoch(self, x, t, seed: int, epoch: int, iter0: int, total_iters: int):
        """One training epoch in one library call (fdtd_mlp_train_epoch):
        seeded shuffled minibatches of x [n, 17] / t [n], loss and gradient,
        Adam with the cosine-decayed rate; returns the epoch's mean batch loss
        as a device FP64 scalar."""
        torch = self.torch
        if not hasattr(self, "tws"):
            self.tws_bytes = self.lib.fdtd_mlp_train_workspace_bytes(self.batch)
            self.tws = torch.empty(self.tws_bytes, dtype=torch.uint8, device=self.dev)
            self.loss_mean = torch.zeros(1, dtype=torch.float64, device=self.dev)
        st = torch.cuda.current_stream(self.dev).cuda_stream
        _check(self.lib, None, self.lib.fdtd_mlp_train_epoch(
            self.p.data_ptr(), self.grad.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), x.data_ptr(), t.data_ptr(),
            x.shape[0], self.batch, int(seed), int(epoch), int(iter0), int(total_iters), float(self.lr),
            self.betas[0], self.betas[1], self.eps, self.loss_mean.data_ptr(), self.tws.data_ptr(), self.tws_bytes,
            st))
        return self.loss_mean

    def step(self, x, t, lr=None):
        self.loss_grad(x, t)
        self.t += 1
        st = self.torch.cuda.current_stream(self.dev).cuda_stream
        _check(self.lib, None, self.lib.fdtd_mlp_adam(self.p.data_ptr(), self.grad.data_ptr(), self.m.data_ptr(),
                                                      self.v.data_ptr(), self.p.numel(), self.t,
                                                      float(self.lr if lr is None else lr), self.betas[0],
                                                      self.betas[1], self.eps, st))
        return self.loss


# ------------------------------------------------------------------ Batch
class Batch:
    """Owns one ``fdtd_batch_t``: many independent 1-D runs (specs in the
    ``fdtd_inputs`` format) advanced by one persistent launch per step call."""

    def __init__(self, specs, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._alloc = _TorchAllocator(self.device)
        n = len(specs)
        arr = (fdtd_run_desc * n)()
        self._keep = []
        for r, sp in enumerate(specs):
            arr[r].grid = _grid_desc(sp["grid"])
            if sp.get("source"):
                arr[r].source = _source_desc(**sp["source"])
            p = sp.get("plasma")
            if p is not None:
                dens = np.ascontiguousarray(p["density"], dtype=np.float64)
                self._keep.append(dens)
                kw = {k: v for k, v in p.items() if k != "density"}
                arr[r].plasma, keep = _plasma_desc(dens.ctypes.data, 0, **kw)
                self._keep.append(keep)
        self.precision = specs[0]["grid"].get("precision", "f32")
        self.f_dtype = (specs[0].get("plasma") or {}).get("f_dtype", "f32")
        rt = fdtd_runtime_desc()
        rt.stream = self.stream.cuda_stream
        rt.alloc, rt.free = self._alloc.alloc_cb, self._alloc.free_cb
        h = ctypes.c_void_p()
        rc = self.lib.fdtd_batch_create(arr, n, ctypes.byref(rt), ctypes.byref(h))
        if rc != FDTD_OK:
            raise FdtdError(rc, self.lib.fdtd_batch_last_error(None).decode())
        self.h = h
        self.nruns = n

    def _check(self, rc):
        if rc != FDTD_OK:
            raise FdtdError(rc, self.lib.fdtd_batch_last_error(self.h).decode())

    def step(self, n: int = 1):
        self._check(self.lib.fdtd_batch_step(self.h, int(n)))

    def info(self) -> dict:
        dt, st, c, nd = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ncl, cc = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.fdtd_batch_info(self.h, ctypes.byref(dt), ctypes.byref(st), ctypes.byref(c),
                                             ctypes.byref(nd), ctypes.byref(ncl), ctypes.byref(cc)))
        return dict(dt=dt.value, steps=st.value, cells=c.value, nodes=nd.value, clusters=ncl.value,
                    cluster_ctas=cc.value)

    def read(self, run: int, name: str):
        """Host numpy copy of one quantity of one run (ex, hy, j, df)."""
        torch = self.torch
        q = QUANTITY[name]
        nb = self.lib.fdtd_batch_quantity_bytes(self.h, int(run), q)
        if name == "df":
            dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[self.f_dtype]
        else:
            dt = torch.float64 if self.precision == "f64" else torch.float32
        out = torch.empty(nb // torch.empty((), dtype=dt).element_size(), dtype=dt)
        if nb:
            self._check(self.lib.fdtd_batch_read(self.h, int(run), q, out.data_ptr(), nb, 0))
        return out.float().numpy() if dt == torch.bfloat16 else out.numpy()

    def autotune(self) -> dict:
        """Time the row-shape candidates on this batch's buffers and keep the fastest (state restored)."""
        vpl, lanes, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
        self._check(self.lib.fdtd_batch_autotune(self.h, ctypes.byref(vpl), ctypes.byref(lanes), ctypes.byref(ms)))
        return {"vpl": vpl.value, "lanes": lanes.value, "ms_per_step": ms.value}

    def write(self, run: int, name: str, values):
        """Overwrite a field (ex: nz+1 values, hy: nz) of one run from host values."""
        q = QUANTITY[name]
        dt = np.float64 if self.precision == "f64" else np.float32
        v = np.ascontiguousarray(np.asarray(values, dtype=dt))
        self._check(self.lib.fdtd_batch_write(self.h, int(run), q, v.ctypes.data, v.nbytes, 0))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fdtd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ Solver
class Solver:
    """Owns one ``fdtd_plasma_t``.  All work runs on the given torch stream."""

    def __init__(self, grid: dict, device: int = 0, stream=None, torch_allocator: bool = True, subdomain=None):
        """subdomain = (offset, extent): the owned planes of the grid's slowest
        axis (fdtd_plasma_create_subdomain); `grid` is then the global grid."""
        import torch
        self.torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.grid = dict(grid)
        g = _grid_desc(grid)
        self._alloc = _TorchAllocator(self.device) if torch_allocator else None
        rt = fdtd_runtime_desc()
        rt.stream = self.stream.cuda_stream
        if self._alloc:
            rt.alloc, rt.free = self._alloc.alloc_cb, self._alloc.free_cb
        rt.alloc_ctx = None
        h = ctypes.c_void_p()
        self.subdomain = None
        if subdomain is None:
            rc = self.lib.fdtd_plasma_create(ctypes.byref(g), ctypes.byref(rt), ctypes.byref(h))
        else:
            axis = int(grid["ndim"]) - 1
            n_global = int(grid["ny"] if axis == 1 else grid["nz"])
            off, ext = int(subdomain[0]), int(subdomain[1])
            sd = fdtd_subdomain_desc(axis, 0, n_global, off, ext)
            rc = self.lib.fdtd_plasma_create_subdomain(ctypes.byref(g), ctypes.byref(sd), ctypes.byref(rt),
                                                       ctypes.byref(h))
            lo, hi = int(off > 0), int(off + ext < n_global)
            self.subdomain = dict(axis=axis, n_global=n_global, offset=off, extent=ext, lo=lo, hi=hi,
                                  origin=off - lo, planes=ext + lo + hi)
        _check(self.lib, None, rc)
        self.h = h
        self.precision = grid.get("precision", "f32")
        self.f_dtype = None

    @classmethod
    def from_spec(cls, spec: dict, device: int = 0, stream=None, subdomain=None) -> "Solver":
        """subdomain = (offset, extent) makes a sub-domain of the spec's grid
        (source and density stay global: the library keeps its part)."""
        s = cls(spec["grid"], device=device, stream=stream, subdomain=subdomain)
        if spec.get("source"):
            s.set_source(**spec["source"])
        if spec.get("plasma") is not None:
            s.set_plasma(**spec["plasma"])
        return s

    # ---- configuration
    def set_source(self, kind="gauss_sine", location="point", amp=1.0, fc=0.0, tau=1.0, t0=0.0,
                   i=0, j=0, k=0, i0=0, i1=0, j0=0, j1=0):
        d = fdtd_source_desc(SRC_KIND[kind], SRC_LOC[location], amp, fc, tau, t0, i, j, k, i0, i1, j0, j1)
        _check(self.lib, self.h, self.lib.fdtd_plasma_set_source(self.h, ctypes.byref(d)))

    def set_plasma(self, density, vgrid="signed1d", nv=64, nv_perp=1, te_ev=1.0, vmax_vth=6.0, nu0=0.0,
                   nu_model="nsv", f_dtype="f32", nonlinear=0, seed=0, f0_model="maxwell", s_table=None,
                   evolve_f0=0, mass_ratio=0.0, tg_ev=0.0):
        """s_table = (speeds, cross-sections) for nu_model "table"; f0_model
        "maxwell" or "druyvesteyn"; evolve_f0 with mass_ratio = m/M and tg_ev
        lets F0 evolve (speed grid)."""
        torch = self.torch
        if isinstance(density, torch.Tensor):
            dens = density.to(self.device, torch.float64).contiguous()
            ptr, on_dev = dens.data_ptr(), 1
        else:
            dens = np.ascontiguousarray(density, dtype=np.float64)
            ptr, on_dev = dens.ctypes.data, 0
        d, keep = _plasma_desc(ptr, on_dev, vgrid, nv, nv_perp, te_ev, vmax_vth, nu0, nu_model, f_dtype, nonlinear,
                               seed, f0_model, s_table, evolve_f0, mass_ratio, tg_ev)
        _check(self.lib, self.h, self.lib.fdtd_plasma_set_plasma(self.h, ctypes.byref(d)))
        del keep
        self.f_dtype = f_dtype

    def set_closure(self, params, e_scale, j_scale, n_scale, rho, n_train_max, beta=0.0, engine="mma"):
        """Install the learned closure (params: torch / numpy FP32, 18945 values)."""
        torch = self.torch
        if isinstance(params, torch.Tensor):
            p = params.detach().to(self.device, torch.float32).contiguous()
            ptr, dev = p.data_ptr(), 1
        else:
            p = np.ascontiguousarray(params, dtype=np.float32)
            ptr, dev = p.ctypes.data, 0
        n = p.numel() if isinstance(p, torch.Tensor) else p.size
        if n != MLP_NPARAMS:
            raise ValueError("closure needs 18945 parameters")
        d = fdtd_closure_desc(ptr, dev, {"mma": 0, "tcgen05": 1}[engine], float(e_scale), float(j_scale),
                              float(n_scale), float(rho), float(n_train_max), float(beta))
        _check(self.lib, self.h, self.lib.fdtd_plasma_set_closure(self.h, ctypes.byref(d)))

    def closure_shape(self):
        a, b = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib, self.h, self.lib.fdtd_plasma_closure_shape(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_recording(self, samples, count, rate, seed=0):
        """Record training samples into the device tensors ``samples`` (float32,
        capacity x 19) and ``count`` (one int64, zeroed by the caller)."""
        cap = samples.numel() // 19
        _check(self.lib, self.h, self.lib.fdtd_plasma_set_recording(self.h, samples.data_ptr(), cap, count.data_ptr(),
                                                                    float(rate), int(seed)))

    # ---- stepping
    def step(self, n: int = 1):
        _check(self.lib, self.h, self.lib.fdtd_plasma_step(self.h, int(n)))

    def step_half(self, half: int):
        """Half 0: H^{n+1/2}; half 1: delta f, J and E^{n+1} (fdtd_plasma_step_half)."""
        _check(self.lib, self.h, self.lib.fdtd_plasma_step_half(self.h, int(half)))

    def halo_bytes(self, which: str) -> int:
        return self.lib.fdtd_plasma_halo_bytes(self.h, HALO[which])

    def halo_pack(self, which: str, out):
        """Copy halo `which` ("e": first owned plane's tangential E, "h": last
        owned plane's tangential H) into the torch tensor `out` (device:
        stream-ordered; host: synchronous)."""
        _check(self.lib, self.h, self.lib.fdtd_plasma_halo_pack(self.h, HALO[which], out.data_ptr(), int(out.is_cuda)))
        return out

    def halo_unpack(self, which: str, buf):
        """Write a neighbour's halo into the ghost plane ("e": above, "h": below)."""
        _check(self.lib, self.h, self.lib.fdtd_plasma_halo_unpack(self.h, HALO[which], buf.data_ptr(), int(buf.is_cuda)))

    def time_kernels(self, n: int) -> dict:
        """Eager, event-timed steps: average ms per launch of each kernel."""
        out = (ctypes.c_double * 5)()
        _check(self.lib, self.h, self.lib.fdtd_plasma_time_kernels(self.h, int(n), out))
        return dict(h=out[0], kinetic=out[1], closure=out[2], e=out[3], step=out[4])

    def autotune(self) -> dict:
        """Time the candidate launch shapes on this handle's buffers and keep
        the fastest (state restored afterwards); see fdtd_plasma_autotune."""
        r = fdtd_tune_result()
        _check(self.lib, self.h, self.lib.fdtd_plasma_autotune(self.h, ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in fdtd_tune_result._fields_}

    def check_canaries(self) -> int:
        """Allocations whose guard bytes changed (needs FDTD_PLASMA_CANARIES=1 at create)."""
        n = ctypes.c_int64(-1)
        _check(self.lib, self.h, self.lib.fdtd_plasma_check_canaries(self.h, ctypes.byref(n)))
        return n.value

    def set_option(self, option: str, value: int):
        """Runtime option: "fused_stencils" (0 / 1, default 0; FDTD_OPT_FUSED_STENCILS),
        "stencil_tz" (0 / planes per block of the TMA column stencils; FDTD_OPT_STENCIL_TZ) or
        "kinetic_shape" (stages * 10**9 + vpl * 10**6 + l * 1000 + bps, 0 = default; FDTD_OPT_KINETIC_SHAPE) or
        "fused_rows" (rows per block of the 2-D fused column march, 0 = the tile kernel; FDTD_OPT_FUSED_ROWS)."""
        code = {"fused_stencils": 1, "stencil_tz": 2, "kinetic_shape": 3, "fused_rows": 4}[option]
        _check(self.lib, self.h, self.lib.fdtd_plasma_set_option(self.h, code, int(value)))

    def launch_shapes(self) -> dict:
        """The launch shapes in use (tuned, cached or default)."""
        r = fdtd_tune_result()
        _check(self.lib, self.h, self.lib.fdtd_plasma_launch_shapes(self.h, ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in fdtd_tune_result._fields_ if not k.endswith("_ms") and k != "reserved"}

    def reset(self):
        _check(self.lib, self.h, self.lib.fdtd_plasma_reset(self.h))

    # ---- I/O
    def quantity_bytes(self, name: str) -> int:
        return self.lib.fdtd_plasma_quantity_bytes(self.h, QUANTITY[name])

    def _dtype(self, name):
        torch = self.torch
        if name in ("df", "f0"):
            return {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[self.f_dtype]
        return torch.float64 if self.precision == "f64" else torch.float32

    def plasma_shape(self):
        ns, nn = ctypes.c_int64(), ctypes.c_int64()
        _check(self.lib, self.h, self.lib.fdtd_plasma_plasma_shape(self.h, ctypes.byref(ns), ctypes.byref(nn)))
        return ns.value, nn.value

    def read(self, name: str, device: bool = True):
        """Quantity as a torch tensor on the device (stream-ordered) or, with
        device=False, as a host numpy array (synchronous)."""
        torch = self.torch
        nb = self.quantity_bytes(name)
        dt = self._dtype(name)
        n = nb // torch.empty((), dtype=dt).element_size()
        if nb == 0:     # no plasma (J, delta f) on this grid or sub-domain
            out = torch.empty((0, self.plasma_shape()[1]) if name in ("df", "f0") else 0, dtype=dt,
                              device=self.device if device else "cpu")
            return out if device else (out.float().numpy() if dt == torch.bfloat16 else out.numpy())
        if device:
            out = torch.empty(n, dtype=dt, device=self.device)
            _check(self.lib, self.h, self.lib.fdtd_plasma_read_fields(self.h, QUANTITY[name], out.data_ptr(), nb, 1))
        else:
            out = torch.empty(n, dtype=dt)
            _check(self.lib, self.h, self.lib.fdtd_plasma_read_fields(self.h, QUANTITY[name], out.data_ptr(), nb, 0))
        if name in ("df", "f0"):
            out = out.view(self.plasma_shape())
        return out if device else (out.float().numpy() if dt == torch.bfloat16 else out.numpy())

    def write(self, name: str, values):
        torch = self.torch
        dt = self._dtype(name)
        if isinstance(values, torch.Tensor):
            t = values.to(self.device, dt).contiguous()
            on_dev = 1
        else:
            t = torch.as_tensor(np.ascontiguousarray(values)).to(dt).contiguous()
            on_dev = 0
        nb = t.numel() * t.element_size()
        _check(self.lib, self.h, self.lib.fdtd_plasma_write_fields(self.h, QUANTITY[name], t.data_ptr(), nb, on_dev))
        if on_dev:
            self.stream.synchronize()

    def info(self):
        dt, n = ctypes.c_double(), ctypes.c_int64()
        _check(self.lib, self.h, self.lib.fdtd_plasma_info(self.h, ctypes.byref(dt), ctypes.byref(n)))
        return dt.value, n.value

    @property
    def dt(self) -> float:
        return self.info()[0]

    def diagnostics(self) -> dict:
        d = fdtd_diag()
        _check(self.lib, self.h, self.lib.fdtd_plasma_diagnostics(self.h, ctypes.byref(d)))
        return dict(energy=d.energy, energy_plain=d.energy_plain, number=d.number,
                    number_max_cell=d.number_max_cell, number_abs=d.number_abs, finite=bool(d.finite), step=d.step)

    def poynting(self, box) -> list:
        """Power out of the box (i0, i1, j0, j1, k0, k1) at the current step:
        [x0, x1, y0, y1, z0, z1, net outward] (FP64)."""
        b = (ctypes.c_int64 * 6)(*[int(v) for v in box])
        out = (ctypes.c_double * 7)()
        _check(self.lib, self.h, self.lib.fdtd_plasma_poynting(self.h, b, out))
        return list(out)

    def set_ports(self, ports, freqs):
        """Running-DFT ports: ports = list of polarisation-node index arrays,
        freqs in Hz; see fdtd_plasma_set_ports."""
        cells = [np.ascontiguousarray(c, dtype=np.int64).ravel() for c in ports]
        off = np.zeros(len(cells) + 1, dtype=np.int64)
        off[1:] = np.cumsum([c.size for c in cells])
        flat = np.concatenate(cells) if cells else np.zeros(1, np.int64)
        fr = np.ascontiguousarray(freqs, dtype=np.float64).ravel()
        i64 = ctypes.POINTER(ctypes.c_int64)
        _check(self.lib, self.h, self.lib.fdtd_plasma_set_ports(
            self.h, len(cells), off.ctypes.data_as(i64), flat.ctypes.data_as(i64), fr.size,
            fr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        self._nports, self._nfreq = len(cells), fr.size

    def port_spectra(self) -> np.ndarray:
        """The port sums X[p, f] (complex128, [nports, nfreq])."""
        out = np.zeros((getattr(self, "_nports", 0), getattr(self, "_nfreq", 0), 2), dtype=np.float64)
        _check(self.lib, self.h, self.lib.fdtd_plasma_read_ports(
            self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.nbytes))
        return out[..., 0] + 1j * out[..., 1]

    def save_state(self, device: bool = True):
        torch = self.torch
        nb = self.lib.fdtd_plasma_state_bytes(self.h)
        buf = torch.empty(nb, dtype=torch.uint8, device=self.device if device else "cpu")
        _check(self.lib, self.h, self.lib.fdtd_plasma_save_state(self.h, buf.data_ptr(), nb, int(device)))
        return buf

    def load_state(self, buf):
        nb = buf.numel()
        _check(self.lib, self.h, self.lib.fdtd_plasma_load_state(self.h, buf.data_ptr(), nb, int(buf.is_cuda)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.fdtd_plasma_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
