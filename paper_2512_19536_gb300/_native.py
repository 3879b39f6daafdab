"""ctypes binding of libpolydg.so (include/polydg.h): argument marshalling only.

Every computation happens in the library's CUDA kernels.  Device vectors are
torch CUDA tensors (float64, contiguous, caller cell order); host arrays are
numpy.  There is no fallback: if the shared library is missing, loading fails
with an error that says how to build it.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpolydg.so")

POLYDG_OK, POLYDG_EINVAL, POLYDG_ENOMEM, POLYDG_ECUDA = 0, -1, -2, -3
POLYDG_ENOTSPD, POLYDG_ENOTCONV, POLYDG_EBREAKDOWN, POLYDG_ENONFINITE = -4, -5, -6, -7
POLYDG_FP64, POLYDG_FP32, POLYDG_BF16 = 0, 1, 2
POLYDG_IONIC_NODAL, POLYDG_IONIC_MODAL = 0, 1
IONIC_FORM = {"nodal": POLYDG_IONIC_NODAL, "modal": POLYDG_IONIC_MODAL}
PRECISION = {"fp64": POLYDG_FP64, "fp32": POLYDG_FP32, "bf16": POLYDG_BF16}

EXPORTS = ["polydg_last_error", "polydg_setup", "polydg_setup3d", "polydg_get_info", "polydg_get_faces",
           "polydg_matvec", "asm_setup", "asm_get_info", "asm_apply", "pcg_solve", "sim_create",
           "monodomain_step", "sim_get_state", "sim_set_potential", "sim_step_index",
           "sim_destroy", "asm_destroy", "polydg_destroy", "polydg_spd_inverse_static",
           "batch_create", "batch_get_groups", "batch_step", "batch_destroy", "guess_n_params",
           "guess_create", "guess_get_params", "guess_set_scales", "guess_propose",
           "guess_train_step", "sim_set_guess", "guess_destroy", "polydg_sym_eig",
           "shared_local_setup", "shared_local_info", "shared_local_apply", "shared_local_destroy",
           "sim_set_shared_local", "asm_autotune", "pcg_solve_trace", "pcg_lanczos_extremes",
           "sim_set_history", "sim_set_ionic_form", "polydg_set_wait_limit", "sim_set_state",
           "sim_get_ionic_coeffs", "sim_get_ionic_aux", "sim_set_ionic_aux"]


class polydg_mesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("vertices", C.POINTER(C.c_double)),
                ("n_cells", C.c_int64), ("cell_ptr", C.POINTER(C.c_int64)),
                ("cell_vtx", C.POINTER(C.c_int32)), ("sigma", C.POINTER(C.c_double))]


class polydg_mesh3d(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("vertices", C.POINTER(C.c_double)),
                ("n_cells", C.c_int64), ("cell_face_ptr", C.POINTER(C.c_int64)),
                ("face_vtx", C.POINTER(C.c_int32)), ("sigma", C.POINTER(C.c_double))]


class polydg_info(C.Structure):
    _fields_ = [("n_cells", C.c_int64), ("n_dofs", C.c_int64), ("n_faces", C.c_int64),
                ("n_blocks", C.c_int64), ("n_nodes", C.c_int64), ("p", C.c_int32),
                ("n_p", C.c_int32), ("n_subdomains", C.c_int32),
                ("max_subdomain_dofs", C.c_int32)]


class pcg_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("status", C.c_int32), ("relres", C.c_double),
                ("bnorm", C.c_double)]


class sim_params(C.Structure):
    _fields_ = [("u0", C.c_double), ("stim_x0", C.c_double), ("stim_y0", C.c_double),
                ("stim_amplitude", C.c_double), ("stim_width", C.c_double),
                ("stim_duration", C.c_double), ("rtol", C.c_double), ("maxit", C.c_int32),
                ("flexible", C.c_int32), ("stim_z0", C.c_double)]


class step_stats(C.Structure):
    _fields_ = [("steps_done", C.c_int64), ("total_iterations", C.c_int64),
                ("max_iterations", C.c_int32), ("status", C.c_int32),
                ("last_relres", C.c_double), ("pcg_seconds", C.c_double),
                ("guesses_taken", C.c_int64)]


class asm_info(C.Structure):
    _fields_ = [("local_store_bytes", C.c_int64), ("coarse_bytes", C.c_int64),
                ("restrict_bytes", C.c_int64), ("n_subdomains", C.c_int32),
                ("n_coarse", C.c_int32), ("precision", C.c_int32), ("grid", C.c_int32),
                ("rows_per_tile", C.c_int32), ("l2_keep_permille", C.c_int32)]


_lib = None


def load() -> C.CDLL:
    """Load libpolydg.so and declare its signatures (raises if it is not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    L.polydg_last_error.restype = C.c_char_p
    L.polydg_setup.argtypes = [C.POINTER(polydg_mesh), i32, C.POINTER(C.c_int32), dbl, dbl, dbl,
                               C.POINTER(vp)]
    L.polydg_setup3d.argtypes = [C.POINTER(polydg_mesh3d), i32, C.POINTER(C.c_int32), dbl, dbl,
                                 dbl, C.POINTER(vp)]
    L.polydg_get_info.argtypes = [vp, C.POINTER(polydg_info)]
    L.polydg_get_faces.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.polydg_matvec.argtypes = [vp, vp, vp, vp]
    L.asm_setup.argtypes = [vp, C.POINTER(C.c_int32), i32, i32, C.POINTER(vp)]
    L.asm_apply.argtypes = [vp, vp, vp, vp]
    L.asm_get_info.argtypes = [vp, C.POINTER(asm_info)]
    L.pcg_solve.argtypes = [vp, vp, vp, vp, dbl, i32, i32, vp, C.POINTER(pcg_stats)]
    L.sim_create.argtypes = [vp, vp, C.POINTER(sim_params), C.POINTER(vp)]
    L.monodomain_step.argtypes = [vp, i32, vp, C.POINTER(step_stats)]
    L.sim_get_state.argtypes = [vp, vp, vp, vp]
    L.sim_set_potential.argtypes = [vp, vp, vp, vp]
    L.sim_set_history.argtypes = [vp, vp, i32, vp]
    L.polydg_spd_inverse_static.argtypes = [vp, i32, i32, i32, vp]
    L.polydg_spd_inverse_static.restype = i32
    L.sim_step_index.argtypes = [vp]
    L.sim_step_index.restype = i64
    L.batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp)]
    L.batch_get_groups.argtypes = [vp, C.POINTER(C.c_int32)]
    L.batch_step.argtypes = [vp, i32, vp, C.POINTER(step_stats), C.POINTER(dbl)]
    for name in ("batch_create", "batch_get_groups", "batch_step"):
        getattr(L, name).restype = i32
    pd_ = C.POINTER(C.c_double)
    L.guess_n_params.argtypes = [i32]
    L.guess_create.argtypes = [i32, pd_, pd_, C.POINTER(vp)]
    L.guess_get_params.argtypes = [vp, pd_, pd_, pd_, C.POINTER(C.c_int64)]
    L.guess_set_scales.argtypes = [vp, pd_]
    L.guess_propose.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.guess_train_step.argtypes = [vp, vp, vp, i64, C.POINTER(C.c_int64), i64, dbl, pd_, vp]
    L.sim_set_guess.argtypes = [vp, vp, i32]
    L.polydg_sym_eig.argtypes = [i32, pd_, pd_, pd_]
    L.polydg_sym_eig.restype = i32
    L.shared_local_setup.argtypes = [vp, i32, C.POINTER(vp)]
    L.shared_local_info.argtypes = [vp, C.POINTER(C.c_int64), pd_]
    L.shared_local_apply.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(vp), pd_, vp]
    for name in ("shared_local_setup", "shared_local_info", "shared_local_apply"):
        getattr(L, name).restype = i32
    L.pcg_solve_trace.argtypes = [vp, vp, vp, vp, dbl, i32, i32, vp, C.POINTER(pcg_stats), pd_, pd_, i32]
    L.pcg_solve_trace.restype = i32
    L.pcg_lanczos_extremes.argtypes = [pd_, pd_, i32, pd_, pd_]
    L.pcg_lanczos_extremes.restype = i32
    L.asm_autotune.argtypes = [vp, i32, i32, pd_]
    L.asm_autotune.restype = i32
    L.sim_set_shared_local.argtypes = [vp, vp]
    L.sim_set_shared_local.restype = i32
    L.sim_set_ionic_form.argtypes = [vp, i32]
    L.sim_set_ionic_form.restype = i32
    L.shared_local_destroy.argtypes = [vp]
    L.shared_local_destroy.restype = None
    L.polydg_set_wait_limit.argtypes = [i64]
    L.polydg_set_wait_limit.restype = i32
    L.sim_set_state.argtypes = [vp, vp, vp, i64, vp]
    L.sim_set_state.restype = i32
    L.sim_get_ionic_coeffs.argtypes = [vp, vp, vp]
    L.sim_get_ionic_coeffs.restype = i32
    for name in ("sim_get_ionic_aux", "sim_set_ionic_aux"):
        getattr(L, name).argtypes = [vp, vp, vp]
        getattr(L, name).restype = i32
    for name in ("guess_n_params", "guess_create", "guess_get_params", "guess_set_scales",
                 "guess_propose", "guess_train_step", "sim_set_guess"):
        getattr(L, name).restype = i32
    for name in ("sim_destroy", "asm_destroy", "polydg_destroy", "batch_destroy", "guess_destroy"):
        getattr(L, name).argtypes = [vp]
        getattr(L, name).restype = None
    for name in ("polydg_setup", "polydg_get_info", "polydg_get_faces", "polydg_matvec",
                 "asm_setup", "asm_get_info", "asm_apply", "pcg_solve", "sim_create", "monodomain_step",
                 "sim_get_state", "sim_set_potential"):
        getattr(L, name).restype = i32
    _lib = L
    return L


class PolyDGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


def _check(status, allow=()):
    if status != POLYDG_OK and status not in allow:
        raise PolyDGError(status, load().polydg_last_error().decode())
    return status


def _ptr(a, dtype):
    return a.ctypes.data_as(C.POINTER(dtype))


def _dev(t):
    """Device pointer of a contiguous float64 CUDA tensor."""
    if not (t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _method(flexible):
    """The PCG variant flag of the C ABI: False/0 standard, True/1 flexible, "pipelined"/2."""
    if flexible == "pipelined" or (not isinstance(flexible, bool) and flexible == 2):
        return 2
    return int(bool(flexible))


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class PolyDG:
    """Handle of a polydg_ctx (assembled K_h on the device)."""

    def __init__(self, handle):
        self.h = handle
        info = polydg_info()
        _check(load().polydg_get_info(self.h, C.byref(info)))
        self.info = info

    @property
    def n_dofs(self):
        return self.info.n_dofs

    def faces(self):
        n = self.info.n_faces
        plus = np.empty(n, np.int64)
        minus = np.empty(n, np.int64)
        _check(load().polydg_get_faces(self.h, _ptr(plus, C.c_int64), _ptr(minus, C.c_int64)))
        return plus, minus

    def matvec(self, x, y, stream=None):
        _check(load().polydg_matvec(self.h, _dev(x), _dev(y), _stream(stream)))

    def close(self):
        if self.h:
            load().polydg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polydg_setup(vertices, cell_ptr, cell_vtx, sigma, p, subdomain_of_cell, chi_cm=1.0,
                 dt=0.1, eta0=10.0) -> PolyDG:
    v = np.ascontiguousarray(vertices, np.float64)
    cp = np.ascontiguousarray(cell_ptr, np.int64)
    cv = np.ascontiguousarray(cell_vtx, np.int32)
    sg = np.ascontiguousarray(sigma, np.float64).reshape(-1)
    sub = np.ascontiguousarray(subdomain_of_cell, np.int32)
    m = polydg_mesh(len(v), _ptr(v, C.c_double), len(cp) - 1, _ptr(cp, C.c_int64),
                    _ptr(cv, C.c_int32), _ptr(sg, C.c_double))
    h = C.c_void_p()
    _check(load().polydg_setup(C.byref(m), int(p), _ptr(sub, C.c_int32), float(chi_cm),
                               float(dt), float(eta0), C.byref(h)))
    return PolyDG(h)


def polydg_setup3d(vertices, cell_face_ptr, face_vtx, sigma, p, subdomain_of_cell, chi_cm=1.0,
                   dt=0.1, eta0=10.0) -> PolyDG:
    """polydg_setup3d on a polyhedral mesh given by outward triangle facets per cell."""
    v = np.ascontiguousarray(vertices, np.float64)
    fp = np.ascontiguousarray(cell_face_ptr, np.int64)
    fv = np.ascontiguousarray(face_vtx, np.int32).reshape(-1)
    sg = np.ascontiguousarray(sigma, np.float64).reshape(-1)
    sub = np.ascontiguousarray(subdomain_of_cell, np.int32)
    m = polydg_mesh3d(len(v), _ptr(v, C.c_double), len(fp) - 1, _ptr(fp, C.c_int64),
                      _ptr(fv, C.c_int32), _ptr(sg, C.c_double))
    h = C.c_void_p()
    _check(load().polydg_setup3d(C.byref(m), int(p), _ptr(sub, C.c_int32), float(chi_cm),
                                 float(dt), float(eta0), C.byref(h)))
    return PolyDG(h)


def setup_mesh(mesh, sigma, p, subdomain_of_cell, chi_cm=1.0, dt=0.1, eta0=10.0) -> PolyDG:
    """polydg_setup or polydg_setup3d, by the mesh's dimension."""
    if getattr(mesh, "dim", 2) == 3:
        return polydg_setup3d(mesh.vertices, mesh.cell_face_ptr, mesh.face_vtx, sigma, p,
                              subdomain_of_cell, chi_cm, dt, eta0)
    return polydg_setup(mesh.vertices, mesh.cell_ptr, mesh.cell_vtx, sigma, p, subdomain_of_cell,
                        chi_cm, dt, eta0)


class ASM:
    """Handle of an asm_ctx (two-level additive Schwarz preconditioner)."""

    def __init__(self, ctx, handle, precision):
        self.ctx, self.h, self.precision = ctx, handle, precision

    def info(self):
        inf = asm_info()
        _check(load().asm_get_info(self.h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in asm_info._fields_}

    def close(self):
        if self.h:
            load().asm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def asm_setup(ctx: PolyDG, coarse_of_cell=None, q=1, precision="fp64") -> ASM:
    h = C.c_void_p()
    if coarse_of_cell is None:
        cptr = None
    else:
        coarse = np.ascontiguousarray(coarse_of_cell, np.int32)
        cptr = _ptr(coarse, C.c_int32)
    _check(load().asm_setup(ctx.h, cptr, int(q), PRECISION[precision], C.byref(h)))
    return ASM(ctx, h, precision)


def asm_autotune(pc: ASM, rounds=3, iterations=60):
    """Re-cut the local-inverse rows over the CTAs by measured per-CTA times; returns the
    speed-up of a PCG iteration (time before / after)."""
    g = C.c_double()
    _check(load().asm_autotune(pc.h, int(rounds), int(iterations), C.byref(g)))
    return g.value


def asm_apply(pc: ASM, r, z, stream=None):
    _check(load().asm_apply(pc.h, _dev(r), _dev(z), _stream(stream)))


def pcg_solve(ctx: PolyDG, pc, b, x, rtol=1e-8, maxit=10000, flexible=False, stream=None,
              allow=(POLYDG_ENOTCONV,)):
    st = pcg_stats()
    status = load().pcg_solve(ctx.h, pc.h if pc is not None else None, _dev(b), _dev(x),
                              float(rtol), int(maxit), _method(flexible), _stream(stream),
                              C.byref(st))
    _check(status, allow)
    return {"iterations": st.iterations, "status": st.status, "relres": st.relres,
            "bnorm": st.bnorm}


def pcg_solve_trace(ctx: PolyDG, pc, b, x, rtol=1e-8, maxit=10000, flexible=False, stream=None,
                    allow=(POLYDG_ENOTCONV,)):
    """pcg_solve that also returns (alphas, betas) of every iteration (numpy arrays)."""
    st = pcg_stats()
    cap = int(maxit)
    al, be = np.zeros(cap), np.zeros(cap)
    status = load().pcg_solve_trace(ctx.h, pc.h if pc is not None else None, _dev(b), _dev(x),
                                    float(rtol), int(maxit), _method(flexible), _stream(stream),
                                    C.byref(st), _ptr(al, C.c_double), _ptr(be, C.c_double), cap)
    _check(status, allow)
    its = st.iterations
    return ({"iterations": its, "status": st.status, "relres": st.relres, "bnorm": st.bnorm},
            al[:its].copy(), be[:max(its - 1, 0)].copy())


def lanczos_extremes(alphas, betas):
    """(lambda_min, lambda_max) of the Lanczos tridiagonal of PCG coefficients."""
    a = np.ascontiguousarray(alphas, np.float64)
    b = np.zeros(max(len(a), 1))
    b[:len(betas)] = betas
    lo, hi = C.c_double(), C.c_double()
    _check(load().pcg_lanczos_extremes(_ptr(a, C.c_double), _ptr(b, C.c_double), len(a),
                                       C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


class Simulation:
    """Handle of a sim_ctx (coupled monodomain + ionic state on the device)."""

    def __init__(self, ctx, pc, handle):
        self.ctx, self.pc, self.h = ctx, pc, handle

    def close(self):
        if self.h:
            load().sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def step_index(self):
        return load().sim_step_index(self.h)


def sim_create(ctx: PolyDG, pc, u0=-67.0, stimulus=None, rtol=1e-8, maxit=10000,
               flexible=False) -> Simulation:
    s = stimulus or {"x0": 0.5, "y0": 0.5, "amplitude": 0.0, "width": 1.0, "duration": 0.0}
    prm = sim_params(float(u0), s["x0"], s["y0"], s["amplitude"], s["width"], s["duration"],
                     float(rtol), int(maxit), _method(flexible), float(s.get("z0", 0.0)))
    h = C.c_void_p()
    _check(load().sim_create(ctx.h, pc.h if pc is not None else None, C.byref(prm), C.byref(h)))
    return Simulation(ctx, pc, h)


def sim_set_ionic_form(sim: Simulation, form="modal"):
    """Ionic state per quadrature node ("nodal", the default) or in the DG basis ("modal");
    chosen before the first step."""
    _check(load().sim_set_ionic_form(sim.h, IONIC_FORM[form]))


def _stats(st):
    return {"steps_done": st.steps_done, "total_iterations": st.total_iterations,
            "max_iterations": st.max_iterations, "status": st.status,
            "last_relres": st.last_relres, "pcg_seconds": st.pcg_seconds,
            "guesses_taken": st.guesses_taken}


def monodomain_step(sim: Simulation, nsteps=1, stream=None):
    st = step_stats()
    _check(load().monodomain_step(sim.h, int(nsteps), _stream(stream), C.byref(st)))
    return _stats(st)


class Batch:
    """Handle of a batch_ctx: simulations advanced together, one batched PCG launch
    per step.  Keeps the Simulation objects alive while the batch exists."""

    def __init__(self, sims, handle):
        self.sims, self.h = list(sims), handle

    def groups(self):
        g = np.zeros(len(self.sims), np.int32)
        _check(load().batch_get_groups(self.h, _ptr(g, C.c_int32)))
        return g

    def close(self):
        if self.h:
            load().batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_create(sims) -> Batch:
    arr = (C.c_void_p * len(sims))(*[s.h for s in sims])
    h = C.c_void_p()
    _check(load().batch_create(arr, len(sims), C.byref(h)))
    return Batch(sims, h)


def batch_step(batch: Batch, nsteps=1, stream=None, allow=()):
    """Advance every simulation nsteps steps; returns (per-simulation statistics,
    device seconds of the batched steps).  Statuses in `allow` do not raise."""
    st = (step_stats * len(batch.sims))()
    sec = C.c_double()
    _check(load().batch_step(batch.h, int(nsteps), _stream(stream), st, C.byref(sec)), allow)
    return [_stats(x) for x in st], sec.value


def sim_get_state(sim: Simulation, u, y=None, stream=None):
    _check(load().sim_get_state(sim.h, _dev(u), _dev(y) if y is not None else None,
                                _stream(stream)))


def sim_set_potential(sim: Simulation, u, uprev=None, stream=None):
    _check(load().sim_set_potential(sim.h, _dev(u), _dev(uprev) if uprev is not None else None,
                                    _stream(stream)))


def sim_set_history(sim: Simulation, hist, stream=None):
    """Restore the last solutions: hist is a CUDA float64 tensor [count, n_dofs] holding
    U^k, U^{k-1}, ... (caller order)."""
    count = int(hist.shape[0])
    _check(load().sim_set_history(sim.h, _dev(hist), count, _stream(stream)))


def sim_set_state(sim: Simulation, k, y=None, Y=None, stream=None):
    """Restore the ionic state (nodal form: y [5, n_nodes]; modal form: Y [5, n_dofs]) and
    the step index k; call before sim_set_history."""
    _check(load().sim_set_state(sim.h, _dev(y) if y is not None else None,
                                _dev(Y) if Y is not None else None, int(k), _stream(stream)))


def sim_get_ionic_coeffs(sim: Simulation, Y, stream=None):
    """Modal form: the DG coefficients of the five ionic states into Y [5, n_dofs]."""
    _check(load().sim_get_ionic_coeffs(sim.h, _dev(Y), _stream(stream)))


def sim_get_ionic_aux(sim: Simulation, aux, stream=None):
    """Nodal form: the per-node functions the update carries (E_Na, E_K, exp(-K_o/5),
    exp((25 - Na_i)/3), u^{k-1}, exp(-u^{k-1}/720)) into aux [6, n_nodes], in
    sim_get_state's node order."""
    _check(load().sim_get_ionic_aux(sim.h, _dev(aux), _stream(stream)))


def sim_set_ionic_aux(sim: Simulation, aux, stream=None):
    """Nodal form: restore the carried functions after sim_set_state and sim_set_history
    (bit-identical resume)."""
    _check(load().sim_set_ionic_aux(sim.h, _dev(aux), _stream(stream)))


def set_wait_limit(polls):
    """Polls of a grid barrier before the persistent kernels give up (< 0: default)."""
    _check(load().polydg_set_wait_limit(int(polls)))


def spd_inverse_static(mats, n, ld, batch, stream=None):
    """In-place inversion of `batch` SPD float64 matrices (order n, leading dimension
    ld) held in the CUDA tensor `mats`, using only the library's fixed static
    workspace: for callers that cannot allocate device memory."""
    if not (mats.is_cuda and mats.is_contiguous() and str(mats.dtype) == "torch.float64"):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    if mats.numel() < batch * n * ld:
        raise ValueError("tensor smaller than batch * n * ld")
    import torch
    with torch.cuda.device(mats.device):      # the call runs on the device holding mats
        if stream is None:
            stream = torch.cuda.current_stream(mats.device)
        _check(load().polydg_spd_inverse_static(C.c_void_p(mats.data_ptr()), int(n), int(ld),
                                                int(batch), _stream(stream)))


class GuessModel:
    """Handle of a guess_model (learned PCG initial guess, include/polydg.h)."""

    def __init__(self, n_p, handle):
        self.n_p, self.h = n_p, handle

    def params(self):
        """(parameters, Adam m, Adam v, Adam steps) as float64 numpy arrays."""
        n = guess_n_params(self.n_p)
        p, m, v = np.empty(n), np.empty(n), np.empty(n)
        t = C.c_int64()
        _check(load().guess_get_params(self.h, _ptr(p, C.c_double), _ptr(m, C.c_double),
                                       _ptr(v, C.c_double), C.byref(t)))
        return p, m, v, t.value

    def set_scales(self, scales):
        sc = np.ascontiguousarray(scales, np.float64)
        _check(load().guess_set_scales(self.h, _ptr(sc, C.c_double)))

    def close(self):
        if self.h:
            load().guess_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def guess_n_params(n_p):
    return _check_count(load().guess_n_params(int(n_p)))


def _check_count(v):
    if v < 0:
        raise PolyDGError(v, load().polydg_last_error().decode())
    return v


def guess_create(n_p, params, scales=None) -> GuessModel:
    p = np.ascontiguousarray(params, np.float64)
    if p.size != guess_n_params(n_p):
        raise ValueError("wrong number of parameters")
    sc = None if scales is None else np.ascontiguousarray(scales, np.float64)
    h = C.c_void_p()
    _check(load().guess_create(int(n_p), _ptr(p, C.c_double),
                               None if sc is None else _ptr(sc, C.c_double), C.byref(h)))
    g = GuessModel(n_p, h)
    g._keep = (p, sc)
    return g


def guess_propose(model: GuessModel, ctx: PolyDG, uk, uk1, uk2, x, stream=None):
    _check(load().guess_propose(model.h, ctx.h, _dev(uk), _dev(uk1), _dev(uk2), _dev(x),
                                _stream(stream)))


def guess_train_step(model: GuessModel, ctx: PolyDG, traj, samples, lr, stream=None):
    """One Adam step; traj is a [n_states, n_dofs] float64 CUDA tensor (caller order),
    samples an [n, 2] int64 array of (state k, caller cell id).  Returns the loss."""
    smp = np.ascontiguousarray(samples, np.int64)
    loss = C.c_double()
    _check(load().guess_train_step(model.h, ctx.h, _dev(traj), int(traj.shape[0]),
                                   _ptr(smp, C.c_int64), int(smp.shape[0]), float(lr),
                                   C.byref(loss), _stream(stream)))
    return loss.value


def sim_set_guess(sim: Simulation, model, policy=0):
    """policy 0: start from the proposal only if its residual is smaller; 1: always;
    2: from U^k + theta (proposal - U^k), theta minimising the residual on that line;
    3: Galerkin projection onto the proposal (if a model is given) and the last
    24 solution increments (model may be None)."""
    _check(load().sim_set_guess(sim.h, model.h if model is not None else None, int(policy)))
    sim.guess = model


def sym_eig(a):
    """(w, Q) of a symmetric matrix on the host: a = Q diag(w) Q^T, w ascending."""
    A = np.array(a, dtype=np.float64, order="C", copy=True)
    n = A.shape[0]
    w = np.empty(n)
    qt = np.empty((n, n))
    _check(load().polydg_sym_eig(int(n), _ptr(A, C.c_double), _ptr(w, C.c_double),
                                 _ptr(qt, C.c_double)))
    return w, qt.T.copy()


class SharedLocal:
    """Handle of a shared_local (local solves shared by scalar-conductivity simulations)."""

    def __init__(self, ctx, handle):
        self.ctx, self.h = ctx, handle

    def info(self):
        b, sref = C.c_int64(), C.c_double()
        _check(load().shared_local_info(self.h, C.byref(b), C.byref(sref)))
        return {"store_bytes": b.value, "sigma_ref": sref.value}

    def close(self):
        if self.h:
            load().shared_local_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def shared_local_setup(ctx: PolyDG, precision="fp32") -> SharedLocal:
    h = C.c_void_p()
    _check(load().shared_local_setup(ctx.h, PRECISION[precision], C.byref(h)))
    return SharedLocal(ctx, h)


def shared_local_apply(sl: SharedLocal, rs, zs, sigmas, stream=None):
    n = len(rs)
    rp = (C.c_void_p * n)(*[_dev(r).value for r in rs])
    zp = (C.c_void_p * n)(*[_dev(z).value for z in zs])
    sg = np.ascontiguousarray(sigmas, np.float64)
    _check(load().shared_local_apply(sl.h, n, rp, zp, _ptr(sg, C.c_double), _stream(stream)))


def sim_set_shared_local(sim: Simulation, sl):
    """Solve this simulation in lockstep with the batch's other users of `sl`."""
    _check(load().sim_set_shared_local(sim.h, sl.h if sl is not None else None))
    sim.shared = sl
