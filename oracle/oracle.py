"""ctypes wrapper of the FP64 CPU oracle (collage_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this
module.  The CUDA library never does.  The shared object is built here with gcc (OpenMP, no
floating-point contraction) into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "collage_oracle.c")
_HDR = os.path.join(_HERE, "collage_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_fp = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc if the shared object is missing or older than its sources."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = not os.path.exists(_LIB) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Opts(C.Structure):
    _fields_ = [("alpha", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("delta", C.c_double), ("tau", C.c_double), ("w_in", C.c_double),
                ("w_out", C.c_double), ("n_dil", C.c_int), ("dil_weight", C.c_double * 8),
                ("pad_px", C.c_double), ("rho_px", C.c_double), ("cull", C.c_int),
                ("force_kind", C.c_int), ("force_x", C.c_double), ("force_y", C.c_double)]


def options(alpha=3e3, beta=8e4, gamma=5e-4, delta=0.0, tau=0.5, w_in=1.0, w_out=100.0,
            n_dil=4, dil_weight=(1.0, 2.0, 3.0, 4.0), pad_px=0.0, rho_px=1.0, cull=1,
            force_kind=0, force_x=0.5, force_y=0.5) -> Opts:
    """Oracle options; the defaults are the weights of Eq. 8 and the readings of Eqs. 5-7."""
    o = Opts()
    o.alpha, o.beta, o.gamma, o.delta = alpha, beta, gamma, delta
    o.tau, o.w_in, o.w_out = tau, w_in, w_out
    o.n_dil = n_dil
    for k in range(8):
        o.dil_weight[k] = dil_weight[k] if k < len(dil_weight) else 0.0
    o.pad_px, o.rho_px, o.cull = pad_px, rho_px, cull
    o.force_kind, o.force_x, o.force_y = force_kind, force_x, force_y
    return o


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    vp = C.c_void_p
    lib.ora_scene_create.restype = vp
    lib.ora_scene_create.argtypes = [C.c_int, _ip, _ip, _fp, _fp, C.c_int, C.c_int, _ip, _fp]
    lib.ora_scene_free.argtypes = [vp]
    lib.ora_n_vertices.argtypes = [vp, C.c_int]
    lib.ora_total_vertices.argtypes = [vp]
    lib.ora_local_vertices.argtypes = [vp, C.c_int, _dp]
    lib.ora_world_vertices.argtypes = [vp, _dp, C.c_int, _dp]
    lib.ora_signed_distance.argtypes = [vp, _dp, C.c_int, C.c_int, _dp, _dp, _ip, _dp]
    lib.ora_container_sd.argtypes = [vp, C.c_int, _dp, _dp]
    opt = C.POINTER(Opts)
    dpn = C.c_void_p  # nullable double*
    lib.ora_render.argtypes = [vp, _dp, C.c_int, opt, dpn, dpn, dpn]
    lib.ora_eval.argtypes = [vp, _dp, C.c_int, opt, dpn, dpn, dpn, dpn]
    lib.ora_adam.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_int, C.c_double, C.c_double,
                             C.c_double, C.c_double, C.c_void_p, C.c_double, C.c_double]
    for name in ("ora_bins", "ora_bins_bruteforce"):
        f = getattr(lib, name)
        f.restype = C.c_long
        f.argtypes = [vp, _fp, C.c_int, C.c_int, C.c_float, C.c_float, _ip, _ip, C.c_long]
    lib.ora_bin_radius.restype = C.c_float
    lib.ora_bin_radius.argtypes = [vp, C.c_int]
    lib.ora_pair_work.restype = C.c_double
    lib.ora_pair_work.argtypes = [vp, _dp, C.c_int, opt]
    lib.ora_metrics.argtypes = [vp, _dp, C.c_int, opt, _dp, _u8p, _u8p]
    lib.ora_uniform_term.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.POINTER(C.c_double), dpn]
    lib.ora_set_threads.restype = C.c_int
    lib.ora_set_threads.argtypes = [C.c_int]
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Scene:
    """Flattened elements and container of one collage problem (see workloads.make_problem)."""

    def __init__(self, prob: dict, segs_per_cubic: int = 16):
        lib = _load()
        self.n = int(len(prob["kind"]))
        kind = np.ascontiguousarray(prob["kind"], np.int32)
        off = np.ascontiguousarray(prob["pt_off"], np.int32)
        for e in range(self.n):
            npt = off[e + 1] - off[e]
            if kind[e] == 0 and (npt < 3 or npt % 3):
                raise ValueError("cubic path needs 3N control points")
            if kind[e] == 1 and npt < 3 or kind[e] == 2 and npt < 2:
                raise ValueError("too few points")
        self._keep = [kind, off, np.ascontiguousarray(prob["pts"], np.float32),
                      np.ascontiguousarray(prob["hw"], np.float32),
                      np.ascontiguousarray(prob["ring_off"], np.int32),
                      np.ascontiguousarray(prob["ring_pts"], np.float32)]
        k = self._keep
        self.h = lib.ora_scene_create(self.n, k[0], k[1], k[2], k[3], segs_per_cubic,
                                      len(k[4]) - 1, k[4], k[5])
        self.lib = lib

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ora_scene_free(self.h)
            self.h = None

    # geometry -------------------------------------------------------------------------------
    def n_vertices(self, e):
        return self.lib.ora_n_vertices(self.h, e)

    def total_vertices(self):
        return self.lib.ora_total_vertices(self.h)

    def local_vertices(self, e):
        out = np.zeros(2 * self.n_vertices(e))
        self.lib.ora_local_vertices(self.h, e, out)
        return out.reshape(-1, 2)

    def world_vertices(self, params, e):
        out = np.zeros(2 * self.n_vertices(e))
        self.lib.ora_world_vertices(self.h, _d(params), e, out)
        return out.reshape(-1, 2)

    def sd(self, params, e, xy):
        xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
        n = len(xy)
        sd, u = np.zeros(n), np.zeros(n)
        seg = np.zeros(n, np.int32)
        self.lib.ora_signed_distance(self.h, _d(params), e, n, xy.reshape(-1), sd, seg, u)
        return sd, seg, u

    def container_sd(self, xy):
        xy = np.ascontiguousarray(xy, np.float64).reshape(-1, 2)
        out = np.zeros(len(xy))
        self.lib.ora_container_sd(self.h, len(xy), xy.reshape(-1), out)
        return out

    # rendering / loss / gradient ------------------------------------------------------------
    def render(self, params, res, opts):
        ihat, atau, covc = (np.zeros(res * res) for _ in range(3))
        self.lib.ora_render(self.h, _d(params), res, C.byref(opts), _ptr(ihat), _ptr(atau),
                            _ptr(covc))
        return ihat.reshape(res, res), atau.reshape(res, res), covc.reshape(res, res)

    def eval(self, params, res, opts, grad=True, grad_v=False):
        terms = np.zeros(5)
        ga = np.zeros(4 * self.n) if grad else None
        gb = np.zeros(4 * self.n) if grad else None
        gv = np.zeros(2 * self.total_vertices()) if grad_v else None
        self.lib.ora_eval(self.h, _d(params), res, C.byref(opts), _ptr(terms), _ptr(ga),
                          _ptr(gb), _ptr(gv))
        out = {"terms": terms}
        if grad:
            out["grad_a"], out["grad_b"] = ga, gb
        if grad_v:
            out["grad_v"] = gv
        return out

    def bins(self, params, res, tile, rho_px=1.0, pad_px=0.0, brute=False):
        p = np.ascontiguousarray(params, np.float32)
        f = self.lib.ora_bins_bruteforce if brute else self.lib.ora_bins
        cap = 1
        dummy_t, dummy_e = np.zeros(1, np.int32), np.zeros(1, np.int32)
        cnt = f(self.h, p, res, tile, rho_px, pad_px, dummy_t, dummy_e, 0)
        t, e = np.zeros(max(cnt, 1), np.int32), np.zeros(max(cnt, 1), np.int32)
        f(self.h, p, res, tile, rho_px, pad_px, t, e, cnt)
        del cap
        return t[:cnt], e[:cnt]

    def bin_radius(self, e):
        return self.lib.ora_bin_radius(self.h, e)

    def metrics(self, params, res, opts):
        """[obj in shape, shape, overlap, obj outside shape, LC, OO, EA, L-nU] (see ora_metrics).
        L-nU (Sec. 6.1) from its definition: for every non-object shape pixel the squared distance
        to the nearest object pixel centre, that pixel found by a nearest-neighbour search over all
        object pixels; the mean, in unit coordinates."""
        out = np.zeros(8)
        obj = np.zeros(res * res, np.uint8)
        shape = np.zeros(res * res, np.uint8)
        self.lib.ora_metrics(self.h, _d(params), res, C.byref(opts), out, obj, shape)
        obj = obj.reshape(res, res).astype(bool)
        free = shape.reshape(res, res).astype(bool) & ~obj
        out[7] = 0.0
        if obj.any() and free.any():
            d2 = nearest_d2(np.argwhere(obj), np.argwhere(free))
            out[7] = float(d2.sum()) / len(d2) / (float(res) * res)
        return out

    def pair_work(self, params, res, opts):
        return self.lib.ora_pair_work(self.h, _d(params), res, C.byref(opts))


def uniform_term(occ, covc, weights, grad=True):
    """The even-distribution term of Eq. 7 on one square image: (L_u, dL_u/dO [R, R] or None).
    occ = O = 1 - Ihat and covc = the container coverage M, both [R, R]; weights[K] are the weights
    of the K box kernels of widths 5 + 6k px."""
    lib = _load()
    occ = np.ascontiguousarray(occ, np.float64)
    covc = np.ascontiguousarray(covc, np.float64)
    R = occ.shape[0]
    assert occ.shape == (R, R) and covc.shape == (R, R)
    w = np.zeros(8)
    w[:len(weights)] = weights
    lu = C.c_double()
    gou = np.zeros((R, R)) if grad else None
    lib.ora_uniform_term(R, len(weights), w, occ.reshape(-1), covc.reshape(-1), C.byref(lu), _ptr(gou))
    return lu.value, gou


def set_threads(n: int) -> int:
    """Threads of the oracle's OpenMP loops (n < 1: all cores); returns the previous setting."""
    return _load().ora_set_threads(n)


def _d(params):
    return np.ascontiguousarray(params, np.float64).reshape(-1)


def adam(params, m, v, g, step, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8, trainable=None,
         s_min=0.05, s_max=20.0):
    """One FP64 Adam step in place on copies; returns (params, m, v)."""
    lib = _load()
    p, m, v = (np.array(x, np.float64).reshape(-1) for x in (params, m, v))
    g = _d(g)
    tr = None if trainable is None else np.ascontiguousarray(trainable, np.uint8)
    lib.ora_adam(len(p) // 4, p, m, v, g, step, lr, b1, b2, eps, _ptr(tr), s_min, s_max)
    return p, m, v


# outline fitting (Sec. 3, "Vector Representation") -------------------------------------------------
def bernstein_weights(segs_per_cubic: int) -> np.ndarray:
    """[segs, 4] cubic Bernstein weights at the samples t = j / segs (j = 0..segs-1) of one curve,
    the flattening of Sec. 3's cubic paths: sample j = sum_r w[j, r] P_r."""
    t = np.arange(segs_per_cubic, dtype=np.float64) / segs_per_cubic
    u = 1.0 - t
    return np.stack([u * u * u, 3.0 * u * u * t, 3.0 * u * t * t, t * t * t], axis=1)


def control_grad(prob: dict, params, res: int, opts, segs_per_cubic: int = 16):
    """dL/d(points) of every element, [n_pts, 2], and the loss terms, for the points of Sec. 3's
    vector representation (cubic control points; polygon and polyline vertices).

    Chain, step by step: ora_eval gives dL/d(world vertex) (unit coordinates); a world vertex is
    t + s R(theta) v (Eq. 2), so dL/dv = s R(theta)^T dL/d(world vertex); a flattened vertex of curve
    c at sample j is sum_r w[j, r] P[3c + r mod 3N] (Bernstein), so each point collects w[j, r] times
    the vertex gradient over the samples it moves; polygon and polyline points are the vertices."""
    sc = Scene(prob, segs_per_cubic)
    out = sc.eval(params, res, opts, grad=False, grad_v=True)
    gv = out["grad_v"].reshape(-1, 2)
    kind = np.asarray(prob["kind"])
    off = np.asarray(prob["pt_off"])
    p = np.asarray(params, np.float64).reshape(-1, 4)
    w = bernstein_weights(segs_per_cubic)
    dpts = np.zeros((int(off[-1]), 2))
    v0 = 0
    for e in range(len(kind)):
        nvert = sc.n_vertices(e)
        ge = gv[v0:v0 + nvert]
        v0 += nvert
        c, s = np.cos(p[e, 2]), np.sin(p[e, 2])
        # s R^T g, R = [[c, -s], [s, c]]
        gl = p[e, 3] * np.stack([c * ge[:, 0] + s * ge[:, 1], -s * ge[:, 0] + c * ge[:, 1]], axis=1)
        npt = int(off[e + 1] - off[e])
        if kind[e] != 0:
            dpts[off[e]:off[e + 1]] = gl
            continue
        for cv in range(npt // 3):
            gc = gl[cv * segs_per_cubic:(cv + 1) * segs_per_cubic]
            for r in range(4):
                k = (3 * cv + r) % npt
                dpts[off[e] + k] += w[:, r] @ gc
    return dpts, out["terms"]


def adam_points(pts, m, v, g, step, lr=1e-2, b1=0.9, b2=0.999, eps=1e-8):
    """One FP64 Adam step (bias-corrected, as for the transforms, without a clamp) on the points;
    returns new (pts, m, v)."""
    pts, m, v, g = (np.array(x, np.float64) for x in (pts, m, v, g))
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    bc1, bc2 = 1.0 - b1 ** step, 1.0 - b2 ** step
    pts = pts - (lr / bc1) * m / (np.sqrt(v) / np.sqrt(bc2) + eps)
    return pts, m, v


def nearest_d2(sites: np.ndarray, queries: np.ndarray) -> np.ndarray:
    """Exact integer squared distance from each query pixel (row, column) to its nearest site
    pixel: a k-d tree nearest-neighbour search (a library primitive) names the nearest site, and
    the squared distance is formed from the integer coordinates (squared distances between
    integer points are exact in double, so the search's choice is a true nearest one; any of
    several equally near sites gives the same value)."""
    from scipy.spatial import cKDTree
    tree = cKDTree(sites.astype(np.float64))
    _, idx = tree.query(queries.astype(np.float64), k=1)
    diff = sites[idx].astype(np.int64) - queries.astype(np.int64)
    return (diff * diff).sum(axis=1)


# skeleton-based initialisation (Sec. 4.1) ---------------------------------------------------------
def medial_axis(covc: np.ndarray):
    """(D2, axis) of a container raster covc [R, R] (Sec. 4.1: the medial axis and the medial width).

    inside = covc >= 1/2, the pixels one step beyond the image outside.  D2 is the squared distance
    in pixels from each inside pixel centre to the nearest outside pixel centre (0 outside), the
    nearest one found by a nearest-neighbour search over every outside pixel (nearest_d2).  The axis
    is the ridge of D2: inside pixels that are a maximum of D2 along one of the four lines through
    them (horizontal, vertical, the two diagonals), D2(p) >= both line neighbours and > at least
    one (neighbours beyond the image count 0)."""
    R = covc.shape[0]
    inside = covc >= 0.5
    ring = [(i, j) for i in range(-1, R + 1) for j in (-1, R)] + [(i, j) for i in (-1, R) for j in range(R)]
    outside = np.concatenate([np.argwhere(~inside), np.array(ring, np.int64)])
    D2 = np.zeros((R, R), np.int64)
    q = np.argwhere(inside)
    if len(q):
        D2[q[:, 0], q[:, 1]] = nearest_d2(outside, q)
    pad = np.zeros((R + 2, R + 2), np.int64)
    pad[1:-1, 1:-1] = D2
    axis = np.zeros((R, R), bool)
    for dx, dy in ((1, 0), (0, 1), (1, 1), (1, -1)):
        a = pad[1 + dy:R + 1 + dy, 1 + dx:R + 1 + dx]
        b = pad[1 - dy:R + 1 - dy, 1 - dx:R + 1 - dx]
        axis |= (D2 >= a) & (D2 >= b) & ((D2 > a) | (D2 > b))
    return D2, axis & (D2 > 0)


def mat_init(prob: dict, params, res: int, opts, segs_per_cubic: int = 16):
    """Initial translations along the medial axis (Sec. 4.1): returns (params [n, 4] float32, D2,
    axis).  The elements in decreasing radius r = (bin radius x s) x res (float32; ties: lower
    index) each take the axis pixel of largest D2 (ties: lower pixel index) whose clearance
    min_j (|p - c_j| - r_j) over the elements placed so far is >= r, else the axis pixel of largest
    clearance (ties: lower pixel index); clearances in float32, |p - c|^2 an exact integer.  The
    translation becomes the pixel centre ((x + 1/2) / res, (y + 1/2) / res) in float32."""
    sc = Scene(prob, segs_per_cubic)
    q = np.asarray(params, np.float32).reshape(-1, 4).copy()
    _, _, covc = sc.render(q.astype(np.float64).reshape(-1), res, opts)
    D2, axis = medial_axis(covc)
    cand = np.flatnonzero(axis.reshape(-1))
    if len(cand) == 0:
        return q, D2, axis
    n = len(q)
    rbin = np.array([sc.bin_radius(e) for e in range(n)], np.float32)
    r = (rbin * q[:, 3]) * np.float32(res)
    cx, cy = cand % res, cand // res
    d2c = D2.reshape(-1)[cand]
    clear = np.full(len(cand), np.finfo(np.float32).max, np.float32)
    placed = np.zeros(n, bool)
    for _ in range(n):
        free = np.flatnonzero(~placed)
        e = free[np.lexsort((free, -r[free].astype(np.float64)))[0]]
        ok = np.flatnonzero(clear >= r[e])
        if len(ok):
            c = ok[np.lexsort((cand[ok], -d2c[ok]))[0]]
        else:
            c = np.lexsort((cand, -clear.astype(np.float64)))[0]
        x, y = cx[c], cy[c]
        q[e, 0] = (np.float32(x) + np.float32(0.5)) / np.float32(res)
        q[e, 1] = (np.float32(y) + np.float32(0.5)) / np.float32(res)
        dist = np.sqrt(((cx - x) ** 2 + (cy - y) ** 2).astype(np.float32)) - r[e]
        clear = np.minimum(clear, dist)
        placed[e] = True
    return q, D2, axis
