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
