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
