"""Write the stored expected values under tests/golden/ using only the oracle (and numpy).

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


def main():
    os.makedirs(GOLDEN, exist_ok=True)
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
