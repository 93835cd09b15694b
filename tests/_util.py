"""Shared helpers of the tests: paired GPU / oracle options and the parity tolerances.

Tolerances (the bar of the parity tests):
  - per-pixel coverage composites (Ihat, A_tau): 1e-5 absolute;
  - each loss term: 1e-5 relative, plus 1e-5 / (w h) absolute (one pixel at the coverage
    tolerance) so that terms that are ~0 compare sensibly;
  - gradients: 1e-3 relative per component, against max(|g_ref|, 1e-2 max_j |g_ref_j|) over the
    same parameter type (tx, ty, theta, s), since near-zero components cannot meet a pure relative
    bound;
  - bins and tile lists: bit-exact.
"""
from __future__ import annotations

import numpy as np

from paper_2406_04008_gb300 import workloads as W

COV_ATOL = 1e-5
LOSS_RTOL = 1e-5
GRAD_RTOL = 1e-3
GRAD_FLOOR = 1e-2

LOSS_KEYS = ("alpha", "beta", "gamma", "delta", "tau", "w_in", "w_out", "pad_px", "rho_px")


def paired(**kw):
    """(GPU option kwargs, oracle options) for the same loss configuration."""
    from oracle import oracle as O
    loss = dict(alpha=3e3, beta=8e4, gamma=5e-4, delta=0.0, tau=0.5, w_in=1.0, w_out=100.0,
                pad_px=0.0, rho_px=1.0, n_dil=4, dil_weight=(1.0, 2.0, 3.0, 4.0),
                force_kind=0, force_x=0.5, force_y=0.5)
    gpu_extra = {}
    for k, v in kw.items():
        if k in loss:
            loss[k] = v
        else:
            gpu_extra[k] = v
    g = dict(alpha=loss["alpha"], beta=loss["beta"], gamma=loss["gamma"],
             delta_down=loss["delta"], tau=loss["tau"], w_in=loss["w_in"], w_out=loss["w_out"],
             pad_px=loss["pad_px"], rho_px=loss["rho_px"], n_dilations=loss["n_dil"],
             dil_weight=list(loss["dil_weight"]), force_kind=loss["force_kind"],
             force_x=loss["force_x"], force_y=loss["force_y"])
    g.update(gpu_extra)
    o = O.options(alpha=loss["alpha"], beta=loss["beta"], gamma=loss["gamma"],
                  delta=loss["delta"], tau=loss["tau"], w_in=loss["w_in"], w_out=loss["w_out"],
                  n_dil=loss["n_dil"], dil_weight=loss["dil_weight"], pad_px=loss["pad_px"],
                  rho_px=loss["rho_px"], force_kind=loss["force_kind"], force_x=loss["force_x"],
                  force_y=loss["force_y"])
    return g, o


def check_terms(gpu, ref, res, weights, use_u=True):
    """gpu, ref: [L_c, L_o, L_u, L_down, L]; weights: (alpha, beta, gamma, delta)."""
    tol = [LOSS_RTOL * abs(ref[k]) + COV_ATOL / (res * res) for k in range(4)]
    # the total inherits the weighted tolerances of its parts
    tol.append(sum(abs(w) * t for w, t in zip(weights, tol)) + LOSS_RTOL * abs(ref[4]))
    for k in [0, 1, 3, 4] + ([2] if use_u else []):
        assert abs(gpu[k] - ref[k]) <= tol[k], (k, gpu[k], ref[k], tol[k])


def grad_errors(g, gr):
    g = np.asarray(g, np.float64).reshape(-1, 4)
    gr = np.asarray(gr, np.float64).reshape(-1, 4)
    out = []
    for c in range(4):
        floor = GRAD_FLOOR * np.abs(gr[:, c]).max()
        if floor == 0.0:
            out.append(np.abs(g[:, c]))
            continue
        out.append(np.abs(g[:, c] - gr[:, c]) / np.maximum(np.abs(gr[:, c]), floor))
    return np.stack(out, 1)


def check_grad(g, gr):
    err = grad_errors(g, gr)
    assert err.max() <= GRAD_RTOL, (err.max(0), np.unravel_index(err.argmax(), err.shape))


def small_case(name):
    """Reduced versions of the five workloads: (problem, option kwargs, grid)."""
    if name == "disks16":
        return W.config_problem(1), dict(gamma=0.0), 128
    if name == "blobs40_ragged":
        return W.config_problem(2, n_elems=40, grid=200), dict(), 200
    if name == "mixed120_pad2":
        return W.config_problem(3, n_elems=120, grid=256), dict(pad_px=2.0), 256
    if name == "open150_force":
        return W.config_problem(5, n_elems=150, grid=240), dict(pad_px=1.0, delta=1e3), 240
    if name == "mixed120_point_force":  # force towards a point (Sec. 5), off-centre
        return (W.config_problem(3, n_elems=120, grid=256),
                dict(pad_px=2.0, delta=300.0, force_kind=1, force_x=0.42, force_y=0.57), 256)
    raise KeyError(name)
