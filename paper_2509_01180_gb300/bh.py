"""Thin Python binding of libbh (ctypes).  Argument marshalling only: every step runs in the library.

Names follow the C ABI in include/bh.h.  Device arrays are torch CUDA tensors (PyTorch provides device
memory and streams only); the library must be built in-tree (``paper_2509_01180_gb300/libbh.so``) and
there is no fallback: a missing library raises.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbh.so")

BH_OK, BH_PENDING = 0, 1
(BH_ERR_ARG, BH_ERR_CUDA, BH_ERR_OOM, BH_ERR_BUDGET, BH_ERR_TIMEOUT, BH_ERR_BUSY,
 BH_ERR_UNSUPPORTED) = -1, -2, -3, -4, -5, -6, -7
BH_MODE_FP32, BH_MODE_BF16_SPLIT = 0, 1
BH_PLAN_MATCH_ONLY = 1
BH_MAX_STAGES = 8
BH_STAGE_ROW = BH_MAX_STAGES + 1

# every symbol include/bh.h declares (checked by the CPU tests)
EXPORTS = ["bh_last_error", "bh_status_string", "bh_version", "bh_basis_roots",
           "bh_plan_create", "bh_plan_destroy", "bh_plan_layout", "bh_plan_info", "bh_plan_gemm", "bh_plan_status",
           "bh_plan_probe_wait", "bh_expand", "bh_expand_noalloc", "bh_score_grad", "bh_score_hess",
           "bh_align_batch", "bh_refine_fp64", "bh_align_shifts_workspace", "bh_align_shifts",
           "bh_grid_create", "bh_grid_destroy", "bh_grid_info", "bh_grid_neighbors", "bh_candidates",
           "bh_wedge_create", "bh_wedge_destroy", "bh_wedge_coeffs", "bh_wedge_norm", "bh_energy", "bh_choose_bands",
           "bh_autotune", "bh_autotune_newton", "bh_random_starts",
           "bh_serve_create", "bh_serve_add_template", "bh_serve_submit", "bh_serve_poll", "bh_serve_wait",
           "bh_serve_pause", "bh_serve_stats", "bh_serve_destroy"]


class BHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


class PlanOpts(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("Lmax", ctypes.c_int), ("lambda_max", ctypes.c_double),
                ("mode", ctypes.c_int), ("max_batch", ctypes.c_int), ("flags", ctypes.c_int)]


class AlignOpts(ctypes.Structure):
    _fields_ = [("group", ctypes.c_int), ("tmpl_index", ctypes.c_void_p), ("n_templates", ctypes.c_int),
                ("start_quat_out", ctypes.c_void_p), ("start_score_out", ctypes.c_void_p),
                ("starts_per_thread", ctypes.c_int), ("refine_fp64", ctypes.c_int), ("newton", ctypes.c_int),
                ("wedge", ctypes.c_void_p), ("dealing", ctypes.c_int), ("stage_table", ctypes.c_void_p)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libbh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2509_01180_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.bh_last_error.restype = ctypes.c_char_p
        L.bh_status_string.restype = ctypes.c_char_p
        L.bh_status_string.argtypes = [i]
        L.bh_version.restype = i
        L.bh_basis_roots.argtypes = [i, d, vp, vp, vp, i]
        L.bh_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(PlanOpts)]
        L.bh_plan_destroy.argtypes = [vp]
        L.bh_plan_layout.argtypes = [vp, vp, vp, vp]
        L.bh_plan_info.argtypes = [vp, ctypes.POINTER(PlanOpts)]
        L.bh_plan_gemm.argtypes = [vp, vp, vp]
        L.bh_plan_status.argtypes = [vp]
        L.bh_plan_probe_wait.argtypes = [vp, vp]
        L.bh_expand.argtypes = [vp, vp, i, vp, vp]
        L.bh_expand_noalloc.argtypes = [vp, vp, i, vp, vp]
        L.bh_score_grad.argtypes = [vp, vp, vp, i, vp, i, i, vp, vp, vp]
        L.bh_score_hess.argtypes = [vp, vp, vp, i, vp, i, i, vp, vp, vp, vp]
        L.bh_align_batch.argtypes = [vp, vp, vp, i, vp, i, vp, i, i, vp, vp, ctypes.POINTER(AlignOpts), vp]
        L.bh_refine_fp64.argtypes = [vp, vp, vp, i, vp, vp, i, i, i, vp, i, vp, vp, vp, vp, vp]
        L.bh_choose_bands.argtypes = [vp, vp, vp, i, i, vp, i, vp, i, i, vp, vp, vp]
        L.bh_grid_create.argtypes = [ctypes.POINTER(vp), vp, i, d]
        L.bh_grid_destroy.argtypes = [vp]
        L.bh_grid_info.argtypes = [vp, vp, vp, vp]
        L.bh_grid_neighbors.argtypes = [vp, vp, vp, ctypes.c_longlong]
        L.bh_candidates.argtypes = [vp, vp, vp, vp, i, i, vp, i, i, vp, vp, vp, vp]
        L.bh_wedge_create.argtypes = [vp, vp, d, i, ctypes.POINTER(vp)]
        L.bh_wedge_destroy.argtypes = [vp]
        L.bh_wedge_coeffs.argtypes = [vp, vp, vp, vp]
        L.bh_wedge_norm.argtypes = [vp, vp, vp, i, i, vp, vp, vp]
        for name in EXPORTS:
            if name not in ("bh_last_error", "bh_status_string"):
                getattr(L, name).restype = i
        _serve_sigs(L)
        _lib = L
    return _lib


def _check(status: int, what: str) -> int:
    if status < 0:
        msg = lib().bh_last_error().decode(errors="replace")
        raise BHError(status, f"{what}: {msg or lib().bh_status_string(status).decode()}")
    return status


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def _stream(stream) -> int:
    if stream is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    return int(getattr(stream, "cuda_stream", stream))


def _need(t, dtype_name: str, numel: int, what: str):
    if t is None:
        raise ValueError(f"{what} is required")
    if not t.is_cuda or not t.is_contiguous() or str(t.dtype) != dtype_name or t.numel() < numel:
        raise ValueError(f"{what}: need a contiguous CUDA {dtype_name} tensor with >= {numel} elements, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")


# ------------------------------------------------------------------ host-only basis data
def bh_basis_roots(Lmax: int, lambda_max: float):
    """(K, lambda, c) of the index set, FP64 on the host (no GPU)."""
    K = np.zeros(Lmax + 1, dtype=np.int32)
    cap = 1 << 16
    lam = np.zeros(cap)
    c = np.zeros(cap)
    _check(lib().bh_basis_roots(Lmax, float(lambda_max), K.ctypes.data, lam.ctypes.data, c.ctypes.data, cap),
           "bh_basis_roots")
    n = int(K.sum())
    return K, lam[:n].copy(), c[:n].copy()


# ------------------------------------------------------------------ plans
class Plan:
    """Owns a bh_plan handle."""

    def __init__(self, handle: int):
        self.handle = handle
        o = PlanOpts()
        _check(lib().bh_plan_info(handle, ctypes.byref(o)), "bh_plan_info")
        self.N, self.Lmax, self.lambda_max, self.mode, self.max_batch = o.N, o.Lmax, o.lambda_max, o.mode, o.max_batch
        self.flags = o.flags
        Nb, V = ctypes.c_int(), ctypes.c_int()
        offs = np.zeros(self.Lmax + 2, dtype=np.int32)
        _check(lib().bh_plan_layout(handle, ctypes.addressof(Nb), ctypes.addressof(V), offs.ctypes.data),
               "bh_plan_layout")
        self.Nb, self.V, self.offsets = Nb.value, V.value, offs
        K, Np = ctypes.c_int(), ctypes.c_int()
        _check(lib().bh_plan_gemm(handle, ctypes.addressof(K), ctypes.addressof(Np)), "bh_plan_gemm")
        self.gemm_K, self.gemm_N = K.value, Np.value  # folded expansion GEMM (fundamental voxels, padded rows)

    def destroy(self):
        if self.handle:
            lib().bh_plan_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def bh_plan_create(N: int, Lmax: int, lambda_max: float = 0.0, mode: int = BH_MODE_FP32, max_batch: int = 0,
                   flags: int = 0) -> Plan:
    o = PlanOpts(N, Lmax, float(lambda_max), mode, max_batch, flags)
    h = ctypes.c_void_p()
    _check(lib().bh_plan_create(ctypes.byref(h), ctypes.byref(o)), "bh_plan_create")
    return Plan(h.value)


def bh_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def bh_plan_layout(plan: Plan):
    return plan.Nb, plan.V, plan.offsets.copy()


# ------------------------------------------------------------------ expansion
def bh_plan_status(plan: Plan) -> None:
    """Raise BHError(BH_ERR_TIMEOUT) if a device wait of the plan's work gave up since the last check."""
    _check(lib().bh_plan_status(plan.handle), "bh_plan_status")


def bh_plan_probe_wait(plan: Plan, stream=None) -> None:
    """Enqueue a probe in which a bounded device wait runs out (about 2 s)."""
    _check(lib().bh_plan_probe_wait(plan.handle, _stream(stream)), "bh_plan_probe_wait")


def bh_expand(plan: Plan, vols, coeffs=None, stream=None):
    """vols: CUDA float32 (B, N, N, N); returns coeffs: CUDA float32 (B, Nb, 2) (complex interleaved)."""
    import torch
    B = vols.shape[0]
    _need(vols, "torch.float32", B * plan.N ** 3, "vols")
    if coeffs is None:
        coeffs = torch.empty((B, plan.Nb, 2), dtype=torch.float32, device=vols.device)
    _need(coeffs, "torch.float32", B * plan.Nb * 2, "coeffs")
    _check(lib().bh_expand(plan.handle, _ptr(vols), B, _ptr(coeffs), _stream(stream)), "bh_expand")
    return coeffs


# ------------------------------------------------------------------ score and gradient
def bh_score_grad(plan: Plan, tmpl, sub, quats, L: int, with_grad: bool = True, stream=None):
    """tmpl (Nb,2), sub (B,Nb,2), quats (B,S,4) CUDA float32 -> score (B,S), grad (B,S,3) or None."""
    import torch
    B, S = quats.shape[0], quats.shape[1]
    _need(tmpl, "torch.float32", plan.Nb * 2, "tmpl")
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    _need(quats, "torch.float32", B * S * 4, "quats")
    score = torch.empty((B, S), dtype=torch.float32, device=sub.device)
    grad = torch.empty((B, S, 3), dtype=torch.float32, device=sub.device) if with_grad else None
    _check(lib().bh_score_grad(plan.handle, _ptr(tmpl), _ptr(sub), B, _ptr(quats), S, L, _ptr(score), _ptr(grad),
                               _stream(stream)), "bh_score_grad")
    return score, grad


def bh_score_hess(plan: Plan, tmpl, sub, quats, L: int, stream=None):
    """Score (B,S), gradient (B,S,3) and Hessian (B,S,3,3) at band L."""
    import torch
    B, S = quats.shape[0], quats.shape[1]
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    _need(quats, "torch.float32", B * S * 4, "quats")
    score = torch.empty((B, S), dtype=torch.float32, device=sub.device)
    grad = torch.empty((B, S, 3), dtype=torch.float32, device=sub.device)
    h6 = torch.empty((B, S, 6), dtype=torch.float32, device=sub.device)
    _check(lib().bh_score_hess(plan.handle, _ptr(tmpl), _ptr(sub), B, _ptr(quats), S, L, _ptr(score), _ptr(grad),
                               _ptr(h6), _stream(stream)), "bh_score_hess")
    idx = torch.tensor([[0, 1, 2], [1, 3, 4], [2, 4, 5]], device=sub.device)
    return score, grad, h6[..., idx]


# ------------------------------------------------------------------ alignment
def bh_align_batch(plan: Plan, tmpl, sub, starts, stages, steps: int, group: int = 0, tmpl_index=None,
                   n_templates: int = 0, per_start: bool = False, quat_out=None, score_out=None, stream=None,
                   refine_fp64: int = 0, starts_per_thread: int = 0, newton: bool = False, wedge=None,
                   stage_table=None, dealing: int = 0):
    """Multi-start marching ascent.  Returns (quat (B,4), score (B,)) [+ (start_quat (B,S,4), start_score (B,S))]."""
    import torch
    B, S = starts.shape[0], starts.shape[1]
    dev = sub.device
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    _need(starts, "torch.float32", B * S * 4, "starts")
    _need(tmpl, "torch.float32", plan.Nb * 2 * max(1, n_templates), "tmpl")
    quat = quat_out if quat_out is not None else torch.empty((B, 4), dtype=torch.float32, device=dev)
    score = score_out if score_out is not None else torch.empty((B,), dtype=torch.float32, device=dev)
    st = (ctypes.c_int * len(stages))(*[int(x) for x in stages])
    o = AlignOpts()
    o.group = group
    o.starts_per_thread = starts_per_thread
    o.refine_fp64 = refine_fp64
    o.newton = int(bool(newton))
    o.dealing = dealing
    o.wedge = wedge.handle if wedge is not None else None
    if stage_table is not None:
        _need(stage_table, "torch.int32", B * BH_STAGE_ROW, "stage_table")
        o.stage_table = _ptr(stage_table)
    sq = ss = None
    if per_start or refine_fp64:
        sq = torch.empty((B, S, 4), dtype=torch.float32, device=dev)
        ss = torch.empty((B, S), dtype=torch.float32, device=dev)
        o.start_quat_out, o.start_score_out = _ptr(sq), _ptr(ss)
    if tmpl_index is not None:
        _need(tmpl_index, "torch.int32", B, "tmpl_index")
        o.tmpl_index, o.n_templates = _ptr(tmpl_index), n_templates
    _check(lib().bh_align_batch(plan.handle, _ptr(tmpl), _ptr(sub), B, _ptr(starts), S, st, len(stages), steps,
                                _ptr(quat), _ptr(score), ctypes.byref(o), _stream(stream)), "bh_align_batch")
    if per_start:
        return quat, score, sq, ss
    return quat, score


def bh_refine_fp64(plan: Plan, tmpl, sub, start_quat, start_score, L: int, K: int, tmpl_index=None,
                   n_templates: int = 0, quat_out=None, score_out=None, score64_out=None, stream=None,
                   stage_table=None):
    """FP64 re-score of the K best starts at band L: returns (quat (B,4), score (B,), score64 (B,) float64)."""
    import torch
    B, S = start_quat.shape[0], start_quat.shape[1]
    dev = sub.device
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    _need(start_quat, "torch.float32", B * S * 4, "start_quat")
    _need(start_score, "torch.float32", B * S, "start_score")
    quat = quat_out if quat_out is not None else torch.empty((B, 4), dtype=torch.float32, device=dev)
    score = score_out if score_out is not None else torch.empty((B,), dtype=torch.float32, device=dev)
    s64 = score64_out if score64_out is not None else torch.empty((B,), dtype=torch.float64, device=dev)
    if tmpl_index is not None:
        _need(tmpl_index, "torch.int32", B, "tmpl_index")
    if stage_table is not None:
        _need(stage_table, "torch.int32", B * BH_STAGE_ROW, "stage_table")
    _check(lib().bh_refine_fp64(plan.handle, _ptr(tmpl), _ptr(sub), B, _ptr(start_quat), _ptr(start_score), S, L, K,
                                _ptr(tmpl_index), n_templates, _ptr(stage_table), _ptr(quat), _ptr(score), _ptr(s64),
                                _stream(stream)), "bh_refine_fp64")
    return quat, score, s64


# ------------------------------------------------------------------ random starts
def bh_random_starts(seed: int, B: int, S: int) -> np.ndarray:
    """(B, S, 4) float32 uniform rotations, SplitMix64 + Shoemake (host)."""
    out = np.empty((B, S, 4), dtype=np.float32)
    _check(lib().bh_random_starts(ctypes.c_uint64(seed), B, S, out.ctypes.data), "bh_random_starts")
    return out


# ------------------------------------------------------------------ serving
def bh_align_shifts(plan: Plan, tmpl, vols, shifts, starts, stages, steps: int, group: int = 0,
                    starts_per_thread: int = 0, stream=None):
    """Shift grid x rotational matching: returns (best shift index (B,), quat (B,4), score (B,))."""
    import torch
    B, S = starts.shape[0], starts.shape[1]
    sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.int32).reshape(-1, 3))
    ns = sh.shape[0]
    _need(vols, "torch.float32", B * plan.N ** 3, "vols")
    _need(starts, "torch.float32", B * S * 4, "starts")
    nbytes = int(lib().bh_align_shifts_workspace(plan.handle, B, ns, S))
    ws = torch.empty((max(nbytes, 256) + 255) // 256 * 256 // 4, dtype=torch.float32, device=vols.device)
    idx = torch.empty((B,), dtype=torch.int32, device=vols.device)
    quat = torch.empty((B, 4), dtype=torch.float32, device=vols.device)
    score = torch.empty((B,), dtype=torch.float32, device=vols.device)
    st = (ctypes.c_int * len(stages))(*[int(x) for x in stages])
    o = AlignOpts()
    o.group, o.starts_per_thread = group, starts_per_thread
    _check(lib().bh_align_shifts(plan.handle, _ptr(tmpl), _ptr(vols), B, sh.ctypes.data, ns, _ptr(starts), S, st,
                                 len(stages), steps, _ptr(ws), ws.numel() * 4, _ptr(idx), _ptr(quat), _ptr(score),
                                 ctypes.byref(o), _stream(stream)), "bh_align_shifts")
    return idx, quat, score


# ------------------------------------------------------------------ candidate starts
class Grid:
    """Owning handle of a rotation grid with its neighbour lists on the device."""

    def __init__(self, handle: int, radius: float):
        self.handle = handle
        self.radius = radius
        n, mx, ne = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _check(lib().bh_grid_info(handle, ctypes.byref(n), ctypes.byref(mx), ctypes.byref(ne)), "bh_grid_info")
        self.n, self.max_neighbors, self.n_edges = n.value, mx.value, ne.value

    def neighbors(self) -> list[np.ndarray]:
        off = np.empty(self.n + 1, dtype=np.int32)
        nb = np.empty(max(1, self.n_edges), dtype=np.int32)
        _check(lib().bh_grid_neighbors(self.handle, off.ctypes.data, nb.ctypes.data, nb.size), "bh_grid_neighbors")
        return [nb[off[i]:off[i + 1]].copy() for i in range(self.n)]

    def destroy(self):
        if self.handle:
            lib().bh_grid_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def bh_grid_create(quats: np.ndarray, radius: float) -> Grid:
    """Upload an (n, 4) rotation grid (w, x, y, z) and build its neighbour lists (geodesic angle <= radius)."""
    q = np.ascontiguousarray(quats, dtype=np.float32).reshape(-1, 4)
    h = ctypes.c_void_p()
    _check(lib().bh_grid_create(ctypes.byref(h), q.ctypes.data, q.shape[0], float(radius)), "bh_grid_create")
    return Grid(h.value, float(radius))


def bh_candidates(plan: Plan, grid: Grid, tmpl, sub, L: int, S: int, tmpl_index=None, n_templates: int = 0,
                  starts_out=None, with_index: bool = False, with_scores: bool = False, stream=None):
    """Candidate starts from local maxima of the band-L score on the grid.  Returns (starts (B,S,4),
    index (B,S) or None, grid scores (B,n) or None)."""
    import torch
    B = sub.shape[0]
    dev = sub.device
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    _need(tmpl, "torch.float32", plan.Nb * 2 * max(1, n_templates), "tmpl")
    starts = starts_out if starts_out is not None else torch.empty((B, S, 4), dtype=torch.float32, device=dev)
    idx = torch.empty((B, S), dtype=torch.int32, device=dev) if with_index else None
    sc = torch.empty((B, grid.n), dtype=torch.float32, device=dev) if with_scores else None
    if tmpl_index is not None:
        _need(tmpl_index, "torch.int32", B, "tmpl_index")
    _check(lib().bh_candidates(plan.handle, grid.handle, _ptr(tmpl), _ptr(sub), B, L, _ptr(tmpl_index), n_templates,
                               S, _ptr(starts), _ptr(idx), _ptr(sc), _stream(stream)), "bh_candidates")
    return starts, idx, sc


# ------------------------------------------------------------------ missing wedge
class Wedge:
    """Owning handle of a missing-wedge norm (bh_wedge_create)."""

    def __init__(self, handle: int, L: int):
        self.handle, self.L = handle, L

    def coeffs(self):
        """(q, w) as lists of (2l+1) complex arrays, and |T(0)|^2 (FP64 host copies)."""
        n = (self.L + 1) ** 2
        q = np.empty(2 * n)
        w = np.empty(2 * n)
        c0 = ctypes.c_double()
        _check(lib().bh_wedge_coeffs(self.handle, q.ctypes.data, w.ctypes.data, ctypes.byref(c0)), "bh_wedge_coeffs")
        qc, wc = q[0::2] + 1j * q[1::2], w[0::2] + 1j * w[1::2]
        return ([qc[l * l:(l + 1) ** 2] for l in range(self.L + 1)], [wc[l * l:(l + 1) ** 2] for l in range(self.L + 1)],
                c0.value)

    def destroy(self):
        if self.handle:
            lib().bh_wedge_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def bh_wedge_create(plan: Plan, tvol: np.ndarray, half_angle_deg: float, L: int) -> Wedge:
    v = np.ascontiguousarray(tvol, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(lib().bh_wedge_create(plan.handle, v.ctypes.data, float(half_angle_deg), int(L), ctypes.byref(h)),
           "bh_wedge_create")
    return Wedge(h.value, int(L))


def bh_wedge_norm(plan: Plan, wedge: Wedge, quats, L: int, stream=None):
    """Dn (S,) and its gradient (S, 3) at S rotations."""
    import torch
    S = quats.shape[0]
    _need(quats, "torch.float32", S * 4, "quats")
    dn = torch.empty((S,), dtype=torch.float32, device=quats.device)
    g = torch.empty((S, 3), dtype=torch.float32, device=quats.device)
    _check(lib().bh_wedge_norm(plan.handle, wedge.handle, _ptr(quats), S, L, _ptr(dn), _ptr(g), _stream(stream)),
           "bh_wedge_norm")
    return dn, g


def bh_energy(plan: Plan, tmpl, sub, L: int, tmpl_index=None, n_templates: int = 0, stream=None):
    """Per-degree energy E_l (B, L+1) of xi^l and the energy ratio Ratio(L') = sum_{l>L'} E_l / sum E_l."""
    import torch
    B = sub.shape[0]
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    e = torch.empty((B, L + 1), dtype=torch.float32, device=sub.device)
    _check(lib().bh_energy(plan.handle, _ptr(tmpl), _ptr(sub), B, L, _ptr(tmpl_index), n_templates, _ptr(e),
                           _stream(stream)), "bh_energy")
    ed = e.double()
    tail = ed.flip(1).cumsum(1).flip(1)
    ratio = torch.cat([tail[:, 1:], torch.zeros_like(tail[:, :1])], 1) / ed.sum(1, keepdim=True).clamp_min(1e-300)
    return e, ratio


def bh_choose_bands(plan: Plan, tmpl, sub, L: int, thresholds, L_min: int = 1, tmpl_index=None,
                    n_templates: int = 0, stage_table=None, with_energy: bool = False, stream=None):
    """Per-subtomogram marching bands from the energy ratio: returns (stage_table (B, BH_STAGE_ROW) int32,
    energy (B, L+1) or None)."""
    import torch
    B = sub.shape[0]
    _need(sub, "torch.float32", B * plan.Nb * 2, "sub")
    thr = np.ascontiguousarray(np.asarray(thresholds, dtype=np.float64))
    tab = stage_table if stage_table is not None else torch.empty((B, BH_STAGE_ROW), dtype=torch.int32,
                                                                   device=sub.device)
    _need(tab, "torch.int32", B * BH_STAGE_ROW, "stage_table")
    e = torch.empty((B, L + 1), dtype=torch.float32, device=sub.device) if with_energy else None
    if tmpl_index is not None:
        _need(tmpl_index, "torch.int32", B, "tmpl_index")
    _check(lib().bh_choose_bands(plan.handle, _ptr(tmpl), _ptr(sub), B, L, _ptr(tmpl_index), n_templates,
                                 thr.ctypes.data, len(thr), L_min, _ptr(tab), _ptr(e), _stream(stream)),
           "bh_choose_bands")
    return tab, e


def stage_rows(table) -> list[list[int]]:
    """Host view of a stage table: the bands of every row."""
    t = table.cpu().numpy() if hasattr(table, "cpu") else np.asarray(table)
    return [[int(x) for x in r[1:1 + int(r[0])]] for r in t]


class TuneResult(ctypes.Structure):
    _fields_ = [("align_group", ctypes.c_int), ("align_starts_per_thread", ctypes.c_int), ("align_ms", ctypes.c_float),
                ("gemm_bn", ctypes.c_int), ("expand_ms", ctypes.c_float), ("align_dealing", ctypes.c_int)]


def bh_autotune(plan: Plan, B: int, S: int, stages, steps: int) -> dict:
    """Time the kernel variants for this shape and keep the fastest in the plan."""
    st = (ctypes.c_int * len(stages))(*[int(x) for x in stages])
    r = TuneResult()
    _check(lib().bh_autotune(plan.handle, B, S, st, len(stages), steps, ctypes.byref(r)), "bh_autotune")
    return {k: getattr(r, k) for k, _ in TuneResult._fields_}


def bh_autotune_newton(plan: Plan, B: int, S: int, stages, steps: int) -> dict:
    """Time the Newton kernel's lanes per start and orbit dealings for this shape and keep the fastest in the plan."""
    st = (ctypes.c_int * len(stages))(*[int(x) for x in stages])
    r = TuneResult()
    _check(lib().bh_autotune_newton(plan.handle, B, S, st, len(stages), steps, ctypes.byref(r)),
           "bh_autotune_newton")
    return {"newton_group": r.align_group, "newton_dealing": r.align_dealing, "newton_ms": r.align_ms}


class ServeOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", ctypes.c_int), ("max_batch", ctypes.c_int),
                ("queue_capacity", ctypes.c_int), ("mode", ctypes.c_int), ("steps", ctypes.c_int),
                ("newton", ctypes.c_int), ("express_slots", ctypes.c_int), ("express_ms", ctypes.c_double),
                ("ingest", ctypes.c_int), ("piece", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("template_id", ctypes.c_int), ("B", ctypes.c_int), ("vols", ctypes.c_void_p), ("S", ctypes.c_int),
                ("starts", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("quat_out", ctypes.c_void_p),
                ("score_out", ctypes.c_void_p)]


class ServeCounters(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("express_batches", ctypes.c_uint64), ("in_place_batches", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("inflight_batches", ctypes.c_uint64),
                ("inflight_bytes", ctypes.c_size_t), ("staging_allocs", ctypes.c_uint64),
                ("launch_ms_total", ctypes.c_double), ("launch_ms_max", ctypes.c_double)]


def _serve_sigs(L):
    vp, i = ctypes.c_void_p, ctypes.c_int
    if getattr(L, "_serve_ready", False):
        return
    L.bh_random_starts.argtypes = [ctypes.c_uint64, i, i, vp]
    L.bh_autotune.argtypes = [vp, i, i, vp, i, i, ctypes.POINTER(TuneResult)]
    L.bh_autotune_newton.argtypes = [vp, i, i, vp, i, i, ctypes.POINTER(TuneResult)]
    L.bh_energy.argtypes = [vp, vp, vp, i, i, vp, i, vp, vp]
    L.bh_align_shifts_workspace.argtypes = [vp, i, i, i]
    L.bh_align_shifts_workspace.restype = ctypes.c_size_t
    L.bh_align_shifts.argtypes = [vp, vp, vp, i, vp, i, vp, i, vp, i, i, vp, ctypes.c_size_t, vp, vp, vp,
                                  ctypes.POINTER(AlignOpts), vp]
    L.bh_serve_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ServeOpts)]
    L.bh_serve_add_template.argtypes = [vp, i, vp, ctypes.POINTER(i)]
    L.bh_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.bh_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
    L.bh_serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.bh_serve_pause.argtypes = [vp, i]
    L.bh_serve_stats.argtypes = [vp, ctypes.POINTER(ServeCounters)]
    L.bh_serve_destroy.argtypes = [vp]
    for n in ("bh_random_starts", "bh_autotune", "bh_energy", "bh_align_shifts", "bh_serve_create",
              "bh_serve_add_template", "bh_serve_submit", "bh_serve_poll", "bh_serve_wait", "bh_serve_pause",
              "bh_serve_stats", "bh_serve_destroy"):
        getattr(L, n).restype = i
    L._serve_ready = True


class Server:
    """Owns a bh_server handle; keeps every request's host arrays alive until it completes."""

    def __init__(self, handle):
        self.handle = handle
        self._live = {}

    def add_template(self, vol: np.ndarray) -> int:
        vol = np.ascontiguousarray(vol, dtype=np.float32)
        tid = ctypes.c_int()
        _check(lib().bh_serve_add_template(self.handle, vol.shape[0], vol.ctypes.data, ctypes.byref(tid)),
               "bh_serve_add_template")
        return tid.value

    def submit(self, template_id: int, vols: np.ndarray, S: int, starts: np.ndarray | None = None, seed: int = 0) -> int:
        """Queue a request; returns its ticket (BHError with BH_ERR_BUDGET / BH_ERR_BUSY / BH_ERR_ARG)."""
        vols = np.ascontiguousarray(vols, dtype=np.float32)
        B = vols.shape[0]
        q = np.zeros((B, 4), dtype=np.float32)
        sc = np.zeros((B,), dtype=np.float32)
        st = None if starts is None else np.ascontiguousarray(starts, dtype=np.float32)
        r = Request(template_id, B, vols.ctypes.data, S, 0 if st is None else st.ctypes.data, seed, q.ctypes.data,
                    sc.ctypes.data)
        t = ctypes.c_uint64()
        _check(lib().bh_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "bh_serve_submit")
        self._live[t.value] = (vols, st, q, sc)
        return t.value

    def poll(self, ticket: int):
        """None while pending, else (quat (B,4), score (B,), latency_ms)."""
        lat = ctypes.c_double()
        st = lib().bh_serve_poll(self.handle, ticket, ctypes.byref(lat))
        if st == BH_PENDING:
            return None
        _check(st, "bh_serve_poll")
        _, _, q, sc = self._live.pop(ticket)
        return q, sc, lat.value

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        lat = ctypes.c_double()
        _check(lib().bh_serve_wait(self.handle, ticket, float(timeout_ms), ctypes.byref(lat)), "bh_serve_wait")
        _, _, q, sc = self._live.pop(ticket)
        return q, sc, lat.value

    def pause(self, paused: bool) -> None:
        _check(lib().bh_serve_pause(self.handle, 1 if paused else 0), "bh_serve_pause")

    def stats(self) -> dict:
        c = ServeCounters()
        _check(lib().bh_serve_stats(self.handle, ctypes.byref(c)), "bh_serve_stats")
        return {k: getattr(c, k) for k, _ in ServeCounters._fields_}

    def destroy(self) -> None:
        if self.handle:
            lib().bh_serve_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def bh_serve_create(hbm_budget_bytes: int = 0, max_inflight: int = 0, max_batch: int = 0, queue_capacity: int = 0,
                    mode: int = BH_MODE_BF16_SPLIT, steps: int = 0, newton: bool = False, express_slots: int = 0,
                    express_ms: float = 0.0, ingest: int = 0, piece: int = 0) -> Server:
    L = lib()
    o = ServeOpts(hbm_budget_bytes, max_inflight, max_batch, queue_capacity, mode, steps, int(bool(newton)),
                  express_slots, express_ms, ingest, piece)
    h = ctypes.c_void_p()
    _check(L.bh_serve_create(ctypes.byref(h), ctypes.byref(o)), "bh_serve_create")
    return Server(h.value)
