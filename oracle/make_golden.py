"""Write the stored expected values under tests/golden/ using only the oracle (and numpy).

boosted_waves.json: the 2-D boosted linear waves of Sec. 4.1.1 (see boosted_waves).

fast_wave_minkowski.json: the right-going fast magnetosonic eigenmode of the 1-D (x) flux
Jacobian at the uniform state rho = 1, p = 1, B = (1, 0.5, 0), v = 0, gamma = 5/3 (the
background of the paper's linear-wave tests, Sec. 4.1.1). With U(P) and F^x(P) from the
oracle, the primitive-space Jacobian A = (dU/dP)^-1 dF/dP is formed by central differences and
diagonalised; its largest eigenvalue is the fast speed and its eigenvector (normalised to
delta rho = 1) the mode shape.

Run:  python -m oracle.make_golden
"""
import json
import os

import numpy as np

import oracle
from paper_2410_09146_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(os.path.dirname(HERE), "tests", "golden")


def fast_wave(gamma=5.0 / 3.0, rho=1.0, press=1.0, B=(1.0, 0.5, 0.0), h=1e-6):
    s = I.linear_wave_setup(8)
    s.gamma_eos = gamma
    p = oracle.params(s)
    P0 = np.array([rho, 0.0, 0.0, 0.0, press / (gamma - 1.0), B[0], B[1], B[2]])
    x = np.zeros((1, 3))

    def UF(P):
        o = oracle.prim2con_points(p, x, P[None])
        return o["U"][0], o["F"][0, 0]

    dU = np.zeros((8, 8)); dF = np.zeros((8, 8))
    for k in range(8):
        e = np.zeros(8); e[k] = h * max(1.0, abs(P0[k]))
        Up, Fp = UF(P0 + e); Um, Fm = UF(P0 - e)
        U2p, F2p = UF(P0 + 2 * e); U2m, F2m = UF(P0 - 2 * e)
        dU[:, k] = (-U2p + 8 * Up - 8 * Um + U2m) / (12 * e[k])
        dF[:, k] = (-F2p + 8 * Fp - 8 * Fm + F2m) / (12 * e[k])
    # B^x has zero flux and zero wave speed: drop it from the eigenproblem to keep A regular.
    keep = [0, 1, 2, 3, 4, 6, 7]
    A = np.linalg.solve(dU[np.ix_(keep, keep)], dF[np.ix_(keep, keep)])
    lam, vec = np.linalg.eig(A)
    lam = lam.real
    k = int(np.argmax(lam))
    v = np.zeros(8)
    v[keep] = vec[:, k].real
    v /= v[0]
    return P0, float(lam[k]), v, sorted(lam.tolist())


def oblique_jacobian(P0, shift, n, gamma=5.0 / 3.0, h=1e-6):
    """Primitive-space flux Jacobian along the unit vector n, A_n = (dU/dP)^-1 (n_x dF^x/dP + n_y dF^y/dP), at the
    uniform state P0 in flat space with the constant shift `shift`, by fourth-order central differences of
    the oracle's U(P) and F^d(P)."""
    s = I.linear_wave_setup(8)
    s.gamma_eos = gamma
    s.shift = tuple(shift)
    p = oracle.params(s)
    x = np.zeros((1, 3))

    def UF(P):
        o = oracle.prim2con_points(p, x, P[None])
        return o["U"][0], n[0] * o["F"][0, 0] + n[1] * o["F"][0, 1] + n[2] * o["F"][0, 2]

    dU = np.zeros((8, 8)); dF = np.zeros((8, 8))
    for k in range(8):
        e = np.zeros(8); e[k] = h * max(1.0, abs(P0[k]))
        Up, Fp = UF(P0 + e); Um, Fm = UF(P0 - e)
        U2p, F2p = UF(P0 + 2 * e); U2m, F2m = UF(P0 - 2 * e)
        dU[:, k] = (-U2p + 8 * Up - 8 * Um + U2m) / (12 * e[k])
        dF[:, k] = (-F2p + 8 * Fp - 8 * Fm + F2m) / (12 * e[k])
    return np.linalg.solve(dU, dF)


def oblique_modes(P0, shift, n, gamma=5.0 / 3.0):
    """Eigen-speeds (ascending) and right eigenvectors (columns, normalised to unit max norm, real) of A_n."""
    lam, vec = np.linalg.eig(oblique_jacobian(P0, shift, n, gamma))
    order = np.argsort(lam.real)
    lam, vec = lam.real[order], vec[:, order].real
    vec /= np.max(np.abs(vec), axis=0)[None]
    return lam, vec


BOOST = (0.617213, 0.617213, 0.0)


def boosted_waves():
    """Sec. 4.1.1: sound, Alfven, slow and fast waves on a 2-D periodic square, flat metric with the coordinate
    boost v_x = v_y = 0.617213 (a constant shift), propagating along the diagonal n = (1, 1, 0)/sqrt(2). Sound:
    rho = 1, P = 1, B = 0. MHD waves: rho = 1, P = 1, B = n + 0.5 t with t = (-1, 1, 0)/sqrt(2) (normal field 1,
    in-plane tangential field 0.5). The right-going mode of each family (in the background's rest frame) is the
    largest eigen-speed of its family; the shifted speeds follow from the unshifted ones by lambda - beta.n."""
    g = 5.0 / 3.0
    n = np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    t = np.array([-1.0, 1.0, 0.0]) / np.sqrt(2.0)
    B = n + 0.5 * t
    hydro = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / (g - 1.0), 0.0, 0.0, 0.0])
    mhd = np.array([1.0, 0.0, 0.0, 0.0, 1.0 / (g - 1.0), B[0], B[1], B[2]])
    bn = float(np.dot(BOOST, n))
    out = {"n": n.tolist(), "shift": list(BOOST), "shift_dot_n": bn, "waves": {}}
    # family -> (background, index in the ascending unshifted spectrum: for MHD fast-, Alfven-, slow-, the two
    # zero-speed modes (entropy and the normal field), slow+, Alfven+, fast+; for hydro sound-, six zero-speed
    # modes, sound+). The shifted mode is the eigenvalue nearest lambda - beta.n (the normal-field mode keeps
    # zero speed under the shift, so the ascending order changes).
    for name, P0, idx in (("sound", hydro, 7), ("alfven", mhd, 6), ("slow", mhd, 5), ("fast", mhd, 7)):
        lam0, _ = oblique_modes(P0, (0.0, 0.0, 0.0), n, g)
        lam, vec = oblique_modes(P0, BOOST, n, g)
        j = int(np.argmin(np.abs(lam - (lam0[idx] - bn))))
        out["waves"][name] = {"background_prims": P0.tolist(), "speed": float(lam[j]),
                              "speed_unshifted": float(lam0[idx]), "eigvec_prims": vec[:, j].tolist(),
                              "spectrum": lam.tolist(), "spectrum_unshifted": lam0.tolist()}
    return out


def main():
    os.makedirs(GOLDEN, exist_ok=True)
    bw = boosted_waves()
    bw["cite"] = "Sec. 4.1.1 (linear waves): 2-D sound, Alfven, slow and fast waves with coordinate boost 0.617213 in x and y"
    bw["written_by"] = "python -m oracle.make_golden (oracle prim->cons and flux Jacobians along n, numpy eig)"
    with open(os.path.join(GOLDEN, "boosted_waves.json"), "w") as f:
        json.dump(bw, f, indent=1)
    P0, lam, v, all_lam = fast_wave()
    out = {
        "cite": "Sec. 4.1.1 (linear waves): fast magnetosonic mode; background as in the 32^3 linear-wave workload",
        "written_by": "python -m oracle.make_golden (oracle prim->cons and flux Jacobian, numpy eig)",
        "background_prims": P0.tolist(),
        "fast_speed": lam,
        "eigvec_prims": v.tolist(),
        "all_speeds": all_lam,
    }
    with open(os.path.join(GOLDEN, "fast_wave_minkowski.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
