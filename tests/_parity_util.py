"""Shared helpers of the GPU parity tests (test code, no product logic)."""
import numpy as np


def ratio_scale(o, system, lat, x, R, ratio_ref):
    """Floating-point scale of every lattice-move ratio of one configuration:
    |exp(dJ)| * sum_m |phi_m(r') Ainv[m][l]|, the magnitude of the terms the
    determinant-ratio dot product sums (at least |ratio| and 1). Rounding in
    any summation order, and in any elimination that forms Ainv, is bounded
    relative to this sum, not to the (possibly cancelled) result."""
    Au, Ad = o.inverses(x)
    C = np.asarray(system.C)
    G = lat.G
    out = np.maximum(1.0, np.abs(ratio_ref))
    for i in range(system.N):
        up = i < system.n_up
        A = Au if up else Ad
        l = i if up else i - system.n_up
        n = system.n_up if up else system.n_dn
        for g in range(G):
            h = lat.a if g == 0 else lat.ap
            for k in range(3):
                e = np.array([R[0 * 3 + k], R[1 * 3 + k], R[2 * 3 + k]])
                for sg in (0, 1):
                    c = ((i * G + g) * 3 + k) * 2 + sg
                    rn = x[i] + (1.0 if sg == 0 else -1.0) * h * e
                    chi = o.ao_values(rn)[0]
                    phi = C[:, :n].T @ chi
                    terms = phi * A[:, l]
                    rdet = terms.sum()
                    if rdet != 0.0:
                        out[c] = max(out[c], np.abs(terms).sum() * abs(ratio_ref[c] / rdet))
    return out


def el_scale(system, x, el_ref):
    """Floating-point scale of local energies: |T| + |V_en| + V_ee + |V_nn|
    for configurations x [W][N][3] with reference local energies el_ref [W],
    T = E_L - V the kinetic part (at least |E_L| and 1). E_L is the sum of
    these terms; near a nucleus of large Z they reach thousands of hartree
    and cancel, and rounding in any evaluation order is bounded relative to
    their magnitudes, not to the (possibly small) sum."""
    x = np.asarray(x, float).reshape(len(el_ref), system.N, 3)
    nuc = np.asarray(system.nuc_xyz, float).reshape(-1, 3)
    Z = np.asarray(system.Z, float)
    v_en = np.zeros(len(el_ref))
    for I in range(len(Z)):
        v_en -= Z[I] * np.sum(1.0 / np.linalg.norm(x - nuc[I], axis=2), axis=1)
    v_ee = np.zeros(len(el_ref))
    if system.ee_on:
        for i in range(system.N):
            for j in range(i + 1, system.N):
                v_ee += 1.0 / np.linalg.norm(x[:, i] - x[:, j], axis=1)
    v_nn = 0.0
    for I in range(len(Z)):
        for J in range(I + 1, len(Z)):
            v_nn += Z[I] * Z[J] / np.linalg.norm(nuc[I] - nuc[J])
    el_ref = np.asarray(el_ref, float)
    kinetic = el_ref - (v_en + v_ee + v_nn)
    return np.maximum.reduce([np.ones_like(el_ref), np.abs(el_ref),
                              np.abs(kinetic) + np.abs(v_en) + v_ee + abs(v_nn)])


# ------------------------------------------------------------------ projection
RTOL = 1e-10
# Double-floats share float's exponent range, and the evaluation's
# exponential returns zero below e^-87 (about 2^-125.5, just above float's
# smallest normal number): a weight p = exp(-x) of Eq. 3 far from the
# nucleus carries an absolute error up to that size in the double-float and
# FP32 modes.
W_ABS = 2.0 ** -125
# A decision whose uniform lies within this distance of a bin edge (relative
# to the quantity it is compared with: tau for the waiting time, b for the
# heat bath, the total weight for a comb tooth) may go either way between
# two correct evaluations; it is the only excuse for a parting.
EDGE = 1e-10

# Entries of the parity report (written at the end of the session by
# conftest.py): one per compared run or evaluation case.
REPORT = []


def record(entry):
    REPORT.append(entry)


def compare_interval(system, gw, ow, margins, rtol=RTOL, edge=EDGE):
    """One interval's populations, GPU (gw) against oracle (ow), as returned
    by walkers(): jump counts and log-weights of every walker before the
    comb, comb parents, positions and local energies after it.

    Returns a dict: ok (everything agrees), the number of decisions the
    oracle took (waiting times, heat-bath choices, comb teeth), how many of
    them lay within edge of a bin edge, the worst errors over the slots that
    agree (relative to max(1, |value|), and for local energies also plainly
    relative to |E_L| and relative to the magnitude of their terms), and for
    a parting the implicated walkers and teeth and whether every one of them
    is excused by a near-edge decision of its own."""
    mw, mc, mt = margins
    W = len(ow["parent"])
    bad_walk = (gw["jumps_pre"] != ow["jumps_pre"]) | (
        np.abs(gw["logw_pre"] - ow["logw_pre"]) > rtol * np.maximum(1.0, np.abs(ow["logw_pre"])))
    same_parent = gw["parent"] == ow["parent"]
    el_sc = el_scale(system, ow["x"], ow["EL"])
    x_err = np.max(np.abs(gw["x"] - ow["x"]) / np.maximum(1.0, np.abs(ow["x"])), axis=(1, 2))
    el_err_sc = np.abs(gw["EL"] - ow["EL"]) / el_sc
    bad_state = (x_err > rtol) | (el_err_sc > rtol)
    walkers = set(np.flatnonzero(bad_walk).tolist())
    walkers |= {int(ow["parent"][t]) for t in np.flatnonzero(bad_state & same_parent)}
    teeth = np.flatnonzero(~same_parent).tolist()
    near_w = mw < edge
    near_t = mt < edge
    info = {
        "ok": not walkers and not teeth,
        "decisions": int(np.sum(ow["jumps_pre"]) + 2 * W),
        "near_edge": int(np.sum(near_w) + np.sum(near_t)),
        "min_margin_walker": float(np.min(mw)), "min_margin_comb": float(mc),
    }
    good = ~bad_state & same_parent
    gw_ok = ~bad_walk
    if np.any(good):
        el = ow["EL"][good]
        info["worst_x_rel"] = float(np.max(x_err[good]))
        info["worst_EL_rel"] = float(np.max(np.abs(gw["EL"][good] - el) / np.abs(el)))
        info["worst_EL_term_scaled"] = float(np.max(el_err_sc[good]))
    if np.any(gw_ok):
        lw = ow["logw_pre"][gw_ok]
        info["worst_logw_rel"] = float(np.max(np.abs(gw["logw_pre"][gw_ok] - lw) / np.maximum(1.0, np.abs(lw))))
    if not info["ok"]:
        info["parted_walkers"] = sorted(walkers)
        info["parted_teeth"] = teeth
        # a walker parts only on its own near-edge decision; a tooth on its
        # own, or because a parted walker changed the weights before it
        info["excused"] = bool(all(near_w[s] for s in walkers) and (walkers or all(near_t[t] for t in teeth)))
    return info


def merge_worst(acc, info):
    for k, v in info.items():
        if k.startswith("worst_"):
            acc[k] = max(acc.get(k, 0.0), v)
        elif k in ("decisions", "near_edge"):
            acc[k] = acc.get(k, 0) + v
        elif k.startswith("min_margin"):
            acc[k] = min(acc.get(k, np.inf), v)


def rate_tolerance(lat, w, scale, rtol=RTOL, w_abs=0.0):
    """Tolerance of every rate T_c = w_c/(2 h_c^2) max(rho_c, 0), candidate
    order electron, grid, axis, sign: rtol times the scale of its weight,
    times its spacing factor, times the floating-point scale of its ratio;
    plus an absolute weight error w_abs (W_ABS in the FP32-pipe modes) times
    the same factors. On the a grid w = p(mid) is an exponential, accurate
    relative to itself; on the a' grid w = 1 - p(mid) inherits the absolute
    rounding of p <= 1, so its scale is max(w, 1 - w) (next to a nucleus
    p -> 1 and w is a small difference of numbers near 1)."""
    P = len(w)
    w = np.asarray(w, float)
    g = (np.arange(P) // 6) % lat.G
    h = np.where(g == 0, lat.a, lat.ap)
    w_scale = np.where(g == 0, w, np.maximum(w, 1.0 - w))
    return (rtol * w_scale + w_abs) / (2.0 * h * h) * scale
