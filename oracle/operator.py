"""Brute-force one-step operator of the MM and modified-HV schemes (arXiv 2309.08068), assembled cell
by cell as a dense affine map f^t = G_t f^{t-1} + b_t.

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only the test suite may import it. It is a second,
independent code path beside ``lbm_oracle.c``. It shares no code or table with it: the vector sets
are rebuilt here from the paper's trigonometric formulas, and every step of the collision is written
as a small matrix acting on one cell's populations. The global operator is then the advection
permutation times the block-diagonal collision. Agreement between the two paths to rounding pins
both against a slip in either. Its matrix also feeds the spectrum pins.

Per cell, in the order of the Appendix B loop body:
  moments       MM: D' = sum f^(0) e, B = sum f^(1) b, rho_c = f_0^(0) + sum f^(0)
                    (eq. MacroscopicFieldsMiller)
                HV: D = sum_i e_i, B = sum_i h_i                   (eq. MacroscopicFieldsHV)
  E and J       MM: E = (D'/eps_r - mu0 J_ext / (4 eps_r)) / (1 + mu0 sigma / (4 eps_r)),
                    J = sigma E + J_ext  (eqs. MacroscopicEMiller, MacorscopicCurrentMiller)
                HV: E = D / eps, J = sigma E + J_ext                        (Appendix B note)
  equilibria    MM: eq. equilibriumsMiller                 HV: eq. equilibriumHV
  collision     MM: f' = 2 f_eq - f; f_0^(0)' = 2 rho_c - f_0^(0); f_0^(1) carried (eq. CollisionMiller)
                HV: e_i' = 2 e_i^eq - e_i + T_i, T_i = -(J . v_i) v_i / 2; h_i' = 2 h_i^eq - h_i
                    (eqs. CollisionHV, SourceTermHV, CollisionmodifiedHV)
  imposition    the moving populations of an imposed cell become f_eq(E_imp(t), B_imp(t), J = 0)
  advection     f^t(x + v_k)[k] = f'(x)[k], periodic on every axis (Sections II and III)

The state vector is the canonical component-major layout of ``oracle.OracleLattice.populations``,
flattened: entry k * n + cell. Lattices up to a few thousand unknowns (dense matrices).
"""
from __future__ import annotations

import numpy as np

MM_Q, HV_Q = 50, 36


def mm_vectors():
    """Velocities v_i^p (eq. VelocitySetMiller), electric vectors e_ij^p (eq.
    ElectromagneticVectorsMiller) and magnetic vectors b_ij^p = v_i^p x e_ij^p, as arrays indexed
    [p, i - 1] and [p, i - 1, j]; p = 0, 1, 2 selects the xy, xz and yz planes."""
    v = np.zeros((3, 4, 3))
    for p in range(3):
        for i in range(1, 5):
            a = (2 * i - 1) * np.pi / 4.0
            c, s = np.sqrt(2.0) * np.cos(a), np.sqrt(2.0) * np.sin(a)
            axes = [(0, 1), (0, 2), (1, 2)][p]
            v[p, i - 1, axes[0]] = c
            v[p, i - 1, axes[1]] = s
    v = np.round(v)  # the formulas give +-1 and 0 up to rounding
    e = np.zeros((3, 4, 2, 3))
    for p in range(3):
        for i in range(1, 5):
            e[p, i - 1, 0] = 0.5 * v[p, (i + 2) % 4]  # e_i0 = v_{[(i+2) mod 4]+1} / 2
            e[p, i - 1, 1] = 0.5 * v[p, i % 4]        # e_i1 = v_{[i mod 4]+1} / 2
    b = np.cross(v[:, :, None, :], e)
    return v, e, b


def hv_velocities():
    """Section III: v1 = +x, v2 = +y, v3 = -x, v4 = -y, v5 = -z, v6 = +z."""
    return np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, -1], [0, 0, 1]], dtype=np.float64)


def _mm_index(r, p, i, j):
    return r * 24 + p * 8 + (i - 1) * 2 + j


def _hv_index(r, i, c):
    return r * 18 + (i - 1) * 3 + c


def mm_population_velocities():
    v, _, _ = mm_vectors()
    vel = np.zeros((MM_Q, 3))
    for r in range(2):
        for p in range(3):
            for i in range(1, 5):
                for j in range(2):
                    vel[_mm_index(r, p, i, j)] = v[p, i - 1]
    return vel


def hv_population_velocities():
    v = hv_velocities()
    vel = np.zeros((HV_Q, 3))
    for r in range(2):
        for i in range(1, 7):
            for c in range(3):
                vel[_hv_index(r, i, c)] = v[i - 1]
    return vel


def mm_cell_map(eps_r, mu_r, sigma, mu0, jext, imposed=None):
    """Affine collision of one MM cell: f' = C f + d. jext is J_ext (3,); imposed is None or
    (E_imp, B_imp). Returns C (50 x 50) and d (50,)."""
    v, e, b = mm_vectors()
    # Moment functionals: rows D'(3), B(3), rho_c(1) acting on the 50 populations.
    mom = np.zeros((7, MM_Q))
    for p in range(3):
        for i in range(1, 5):
            for j in range(2):
                k0, k1 = _mm_index(0, p, i, j), _mm_index(1, p, i, j)
                mom[0:3, k0] = e[p, i - 1, j]
                mom[3:6, k1] = b[p, i - 1, j]
                mom[6, k0] = 1.0
    mom[6, 48] = 1.0
    # E = aE D' + cE, J = sigma E + J_ext
    den = 1.0 + mu0 * sigma / (4.0 * eps_r)
    aE = 1.0 / (eps_r * den)
    cE = -mu0 * np.asarray(jext, dtype=np.float64) / (4.0 * eps_r * den)

    def eq_rows(e_coef, b_coef, E_lin, E_const, B_lin, B_const, J_lin, J_const):
        """Equilibria of the 48 moving populations, each a linear map of the 7 moments plus a
        constant: f_eq = v.J/16 + e_coef E.e + b_coef B.b."""
        lin = np.zeros((48, 7))
        const = np.zeros(48)
        for r in range(2):
            for p in range(3):
                for i in range(1, 5):
                    for j in range(2):
                        k = _mm_index(r, p, i, j)
                        vv, ee, bb = v[p, i - 1], e[p, i - 1, j], b[p, i - 1, j]
                        ec = e_coef[r]
                        bc = b_coef[r]
                        lin[k] = vv @ J_lin / 16.0 + ec * (ee @ E_lin) + bc * (bb @ B_lin)
                        const[k] = vv @ J_const / 16.0 + ec * (ee @ E_const) + bc * (bb @ B_const)
        return lin, const

    e_coef = (eps_r / 4.0, 1.0 / 4.0)
    b_coef = (1.0 / (8.0 * mu_r), 1.0 / 8.0)
    E_lin = np.zeros((3, 7))
    E_lin[:, 0:3] = aE * np.eye(3)
    B_lin = np.zeros((3, 7))
    B_lin[:, 3:6] = np.eye(3)
    J_lin = sigma * E_lin
    J_const = sigma * cE + np.asarray(jext, dtype=np.float64)
    lin, const = eq_rows(e_coef, b_coef, E_lin, cE, B_lin, np.zeros(3), J_lin, J_const)
    C = np.zeros((MM_Q, MM_Q))
    d = np.zeros(MM_Q)
    C[:48] = 2.0 * lin @ mom - np.eye(MM_Q)[:48]
    d[:48] = 2.0 * const
    C[48] = 2.0 * mom[6] - np.eye(MM_Q)[48]  # f_0^(0)' = 2 rho_c - f_0^(0)
    C[49, 49] = 1.0                          # f_0^(1) carried
    if imposed is not None:
        E_imp, B_imp = (np.asarray(a, dtype=np.float64) for a in imposed)
        zero = np.zeros((3, 7))
        _, const_imp = eq_rows(e_coef, b_coef, zero, E_imp, zero, B_imp, zero, np.zeros(3))
        C[:48] = 0.0
        d[:48] = const_imp
    return C, d


def _cross_matrix(u):
    """[u]_x with [u]_x a = u x a."""
    return np.array([[0.0, -u[2], u[1]], [u[2], 0.0, -u[0]], [-u[1], u[0], 0.0]])


def hv_cell_map(eps_r, mu_r, sigma, eps0, mu0, jext, imposed=None):
    """Affine collision of one HV cell: f' = C f + d (36 x 36, 36)."""
    vs = hv_velocities()
    eps, mu = eps0 * eps_r, mu0 * mu_r
    sumD = np.zeros((3, HV_Q))
    sumB = np.zeros((3, HV_Q))
    for i in range(1, 7):
        for c in range(3):
            sumD[c, _hv_index(0, i, c)] = 1.0
            sumB[c, _hv_index(1, i, c)] = 1.0
    jext = np.asarray(jext, dtype=np.float64)
    C = -np.eye(HV_Q)
    d = np.zeros(HV_Q)
    for i in range(1, 7):
        vi = vs[i - 1]
        X = _cross_matrix(vi)
        rows_e = [_hv_index(0, i, c) for c in range(3)]
        rows_h = [_hv_index(1, i, c) for c in range(3)]
        # e_i^eq = (D - 3 v_i x B / mu) / 6, h_i^eq = (B + 3 v_i x D / eps) / 6
        e_eq = (sumD - 3.0 * X @ sumB / mu) / 6.0
        h_eq = (sumB + 3.0 * X @ sumD / eps) / 6.0
        # T_i = -(J . v_i) v_i / 2 with J = sigma D / eps + J_ext
        T_lin = -0.5 * np.outer(vi, vi) @ (sigma * sumD / eps)
        T_const = -0.5 * vi * (vi @ jext)
        C[rows_e] += 2.0 * e_eq + T_lin
        d[rows_e] += T_const
        C[rows_h] += 2.0 * h_eq
    if imposed is not None:
        E_imp, B_imp = (np.asarray(a, dtype=np.float64) for a in imposed)
        D_imp = eps * E_imp
        C[:] = 0.0
        for i in range(1, 7):
            X = _cross_matrix(vs[i - 1])
            d[[_hv_index(0, i, c) for c in range(3)]] = (D_imp - 3.0 * X @ B_imp / mu) / 6.0
            d[[_hv_index(1, i, c) for c in range(3)]] = (B_imp + 3.0 * X @ D_imp / eps) / 6.0
    return C, d


def time_value(fn, t):
    """s(t) of a ``workloads.TimeFunction`` at integer time t: sin, table (zero outside) or const."""
    if fn.kind == "sin":
        return fn.amplitude * np.sin(2.0 * np.pi * t / fn.period + fn.phase)
    if fn.kind == "table":
        tab = np.asarray(fn.table, dtype=np.float64).reshape(-1)
        return fn.amplitude * tab[t] if 0 <= t < tab.size else 0.0
    return fn.amplitude


def step_operator(model, shape, t, eps_r=None, mu_r=None, sigma=None, sources=(), eps0=None, mu0=None):
    """The dense affine map of iteration t (state t - 1 -> state t): returns (G, b) with
    f^t = G f^{t-1} + b on the flattened canonical layout. ``sources`` are ``workloads.Source``
    objects; iteration t evaluates them at s(t) (Appendix B loop, t = 1 .. t_max)."""
    nx, ny, nz = (int(s) for s in shape)
    n = nx * ny * nz
    q = MM_Q if model == "mm" else HV_Q
    if eps0 is None:
        eps0 = 1.0 if model == "mm" else 3.0
    if mu0 is None:
        mu0 = 2.0 if model == "mm" else 3.0
    er = np.ones(n) if eps_r is None else np.asarray(eps_r, dtype=np.float64).reshape(-1)
    mr = np.ones(n) if mu_r is None else np.asarray(mu_r, dtype=np.float64).reshape(-1)
    sg = np.zeros(n) if sigma is None else np.asarray(sigma, dtype=np.float64).reshape(-1)
    jext = np.zeros((n, 3))
    e_imp = np.zeros((n, 3))
    b_imp = np.zeros((n, 3))
    imposed = np.zeros(n, dtype=bool)
    for s in sources:
        st = time_value(s.fn, t)
        cells = np.asarray(s.cells, dtype=np.int64).reshape(-1)
        for m, x in enumerate(cells):
            if s.kind == "current":
                jext[x] += np.asarray(s.w, dtype=np.float64)[m] * st
            else:
                e_imp[x] += np.asarray(s.E0, dtype=np.float64) * st
                b_imp[x] += np.asarray(s.B0, dtype=np.float64) * st
                imposed[x] = True
    vel = mm_population_velocities() if model == "mm" else hv_population_velocities()
    N = q * n
    G = np.zeros((N, N))
    b = np.zeros(N)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                c = x + nx * (y + ny * z)
                imp = (e_imp[c], b_imp[c]) if imposed[c] else None
                if model == "mm":
                    C, d = mm_cell_map(er[c], mr[c], sg[c], mu0, jext[c], imp)
                else:
                    C, d = hv_cell_map(er[c], mr[c], sg[c], eps0, mu0, jext[c], imp)
                for k in range(q):
                    vx, vy, vz = (int(a) for a in vel[k])
                    dst = (x + vx) % nx + nx * (((y + vy) % ny) + ny * ((z + vz) % nz))
                    row = k * n + dst
                    G[row, np.arange(q) * n + c] = C[k]
                    b[row] = d[k]
    return G, b
