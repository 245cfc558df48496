"""Deterministic reference solutions that pin the Monte Carlo oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/oracle.py``).

* ``slab_solution``: the gray slab between black walls (the steady limit of
  Eq. 1 with isotropic scattering, Eq. 4 estimators) is the classical
  conservative-scattering slab of radiative transfer.  With optical
  coordinate tau = x / Lambda and thickness tau_L = L / Lambda, the
  non-dimensional emissive function phi = (T - T_cold) / (T_hot - T_cold)
  obeys

      phi(tau) = 1/2 [ E2(tau) + int_0^tau_L phi(t) E1(|tau - t|) dt ]

  and the non-dimensional heat flux is Psi = 1 - 2 int_0^tau_L phi E2 dt.
  It is solved here by product-integration collocation with piecewise-linear
  phi (exact panel integrals through E2, E3, E4) and Richardson
  extrapolation in the panel count.
* ``fuchs_sondheimer``: in-plane conductivity suppression of a film with
  diffuse walls (the analytic thin-film solution, last section of the paper),
  S(delta) = 1 - 3/(2 delta) int_1^inf (t^-3 - t^-5)(1 - exp(-delta t)) dt,
  delta = L / Lambda, evaluated in closed form through E3 and E5 and
  independently by quadrature of the first-flight integral over directions.
* ``mode_table``: per-mode (omega, v, tau, C) of the isotropic quadratic
  dispersion, written with numpy independently of the C oracle.
* ``kappa_bulk`` and ``kappa_film``: (1/3) sum_b C_b v_b^2 tau_b [S(L/Lambda_b)].
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, special

HBAR = 1.054571817e-34
KB = 1.380649e-23


def En(n, x):
    return special.expn(n, np.asarray(x, dtype=np.float64))


# --------------------------------------------------------------------------
# Gray slab
# --------------------------------------------------------------------------
def _F0(s):  # antiderivative of E1
    return -En(2, s)


def _F1(s):  # antiderivative of s E1(s)
    return -s * En(2, s) - En(3, s)


def _lin_E1(a, b, alpha, beta, ti):
    """int_a^b (alpha + beta t) E1(|ti - t|) dt for a <= b (vectorised in ti)."""
    ti = np.asarray(ti, dtype=np.float64)
    out = np.zeros_like(ti)
    c = alpha + beta * ti
    # part of [a, b] right of ti
    ra = np.maximum(a, ti)
    rb = np.maximum(b, ti)
    sa, sb = ra - ti, rb - ti
    out += c * (_F0(sb) - _F0(sa)) + beta * (_F1(sb) - _F1(sa))
    # part of [a, b] left of ti
    la = np.minimum(a, ti)
    lb = np.minimum(b, ti)
    sa, sb = ti - la, ti - lb
    out += c * (_F0(sa) - _F0(sb)) - beta * (_F1(sa) - _F1(sb))
    return out


def _solve_slab(tau_L, M):
    h = tau_L / M
    nodes = np.linspace(0.0, tau_L, M + 1)
    W = np.zeros((M + 1, M + 1))
    for j in range(M + 1):
        if j > 0:  # rising part on [t_{j-1}, t_j]: (t - t_{j-1}) / h
            a, b = nodes[j - 1], nodes[j]
            W[:, j] += _lin_E1(a, b, -a / h, 1.0 / h, nodes)
        if j < M:  # falling part on [t_j, t_{j+1}]: (t_{j+1} - t) / h
            a, b = nodes[j], nodes[j + 1]
            W[:, j] += _lin_E1(a, b, b / h, -1.0 / h, nodes)
    A = np.eye(M + 1) - 0.5 * W
    rhs = 0.5 * En(2, nodes)
    phi = np.linalg.solve(A, rhs)
    return nodes, phi


def _int_lin_E2(a, b, alpha, beta, shift=0.0, sign=1.0):
    """int_a^b (alpha + beta t) E2(sign (t - shift)) dt with sign (t - shift) >= 0."""
    if sign > 0:
        sa, sb = a - shift, b - shift
        G0 = lambda s: -En(3, s)
        G1 = lambda s: -s * En(3, s) - En(4, s)
        c = alpha + beta * shift
        return c * (G0(sb) - G0(sa)) + beta * (G1(sb) - G1(sa))
    sa, sb = shift - a, shift - b  # sa >= sb
    G0 = lambda s: -En(3, s)
    G1 = lambda s: -s * En(3, s) - En(4, s)
    c = alpha + beta * shift
    return c * (G0(sa) - G0(sb)) - beta * (G1(sa) - G1(sb))


def _flux_at(nodes, phi, tau):
    """Non-dimensional flux q*(tau) = 2 E3(tau) + 2 int_0^tau phi E2(tau-t) dt
    - 2 int_tau^tau_L phi E2(t - tau) dt (cold wall phi = 0)."""
    tau_L = nodes[-1]
    q = 2.0 * float(En(3, tau))
    for j in range(len(nodes) - 1):
        a, b = nodes[j], nodes[j + 1]
        h = b - a
        beta = (phi[j + 1] - phi[j]) / h
        alpha = phi[j] - beta * a
        if b <= tau:
            q += 2.0 * float(_int_lin_E2(a, b, alpha, beta, shift=tau, sign=-1.0))
        elif a >= tau:
            q -= 2.0 * float(_int_lin_E2(a, b, alpha, beta, shift=tau, sign=+1.0))
        else:
            q += 2.0 * float(_int_lin_E2(a, tau, alpha, beta, shift=tau, sign=-1.0))
            q -= 2.0 * float(_int_lin_E2(tau, b, alpha, beta, shift=tau, sign=+1.0))
    return q


def _psi(nodes, phi):
    return _flux_at(nodes, phi, 0.0)


def _bin_means(nodes, phi, n_bins):
    """Bin averages of the piecewise-linear phi over n_bins equal bins."""
    tau_L = nodes[-1]
    edges = np.linspace(0.0, tau_L, n_bins + 1)
    out = np.zeros(n_bins)
    for k in range(n_bins):
        xs = np.linspace(edges[k], edges[k + 1], 2001)
        out[k] = np.trapezoid(np.interp(xs, nodes, phi), xs) / (edges[k + 1] - edges[k])
    return out


def slab_solution(tau_L, n_bins=50, M=400, richardson=True):
    """Psi and the bin-averaged phi of the gray slab of optical thickness tau_L.

    Returns dict(psi, phi_bins, T_bins) with T_bins = 2 phi - 1, the
    temperature in units of the wall excess (walls at T_eq +/- dT)."""
    M1 = max(M - M % n_bins, n_bins)
    n1, p1 = _solve_slab(tau_L, M1)
    psi1 = _psi(n1, p1)
    b1 = _bin_means(n1, p1, n_bins)
    if not richardson:
        return {"psi": psi1, "phi_bins": b1, "T_bins": 2 * b1 - 1, "nodes": n1, "phi": p1}
    n2, p2 = _solve_slab(tau_L, 2 * M1)
    psi2 = _psi(n2, p2)
    b2 = _bin_means(n2, p2, n_bins)
    psi = (4 * psi2 - psi1) / 3
    b = (4 * b2 - b1) / 3
    return {"psi": psi, "phi_bins": b, "T_bins": 2 * b - 1, "nodes": n2, "phi": p2,
            "psi_coarse": psi1, "psi_fine": psi2}


def slab_flux_profile(tau_L, taus, M=400):
    """q*(tau) at interior points; constant (= Psi) for the exact solution."""
    nodes, phi = _solve_slab(tau_L, M)
    return np.array([_flux_at(nodes, phi, t) for t in taus])


# --------------------------------------------------------------------------
# Thin film with diffuse walls
# --------------------------------------------------------------------------
def fuchs_sondheimer(delta):
    """S(delta) in closed form: int_1^inf t^-n exp(-delta t) dt = E_n(delta)."""
    d = np.asarray(delta, dtype=np.float64)
    return 1.0 - 1.5 / d * (0.25 - En(3, d) + En(5, d))


def fuchs_sondheimer_quadrature(delta):
    """S(delta) from the first-flight integral of a particle emitted uniformly
    across the film with a |cos| law about the in-plane axis z:
    S = 3/2 int_0^1 (1 - mu^2) g(mu) dmu, mu = |Omega_x|,
    g(mu) = 1 - (mu/delta)(1 - exp(-delta/mu))."""
    def g(mu):
        if mu <= 0.0:
            return 1.0
        return 1.0 - (mu / delta) * (-math.expm1(-delta / mu))
    val, _ = integrate.quad(lambda mu: (1 - mu * mu) * g(mu), 0.0, 1.0, limit=400, epsabs=1e-14)
    return 1.5 * val


def fuchs_sondheimer_specular(delta, p):
    """S(delta, p) for walls that reflect specularly with probability p and
    diffusely otherwise, from the first-flight picture: a particle emitted
    uniformly across the film keeps its in-plane velocity through specular
    reflections and loses it (in expectation) at its first diffuse event, so
    with mu = |Omega_x| its mean path to that event is Lambda g_p(mu),
    g_p(mu) = 1 - (1 - p)(mu/delta)(1 - e^{-delta/mu}) / (1 - p e^{-delta/mu}),
    and S = 3/2 int_0^1 (1 - mu^2) g_p(mu) dmu."""
    def g(mu):
        if mu <= 0.0:
            return 1.0
        e = math.exp(-delta / mu)
        return 1.0 - (1.0 - p) * (mu / delta) * (-math.expm1(-delta / mu)) / (1.0 - p * e)
    val, _ = integrate.quad(lambda mu: (1 - mu * mu) * g(mu), 0.0, 1.0, limit=400, epsabs=1e-14)
    return 1.5 * val


def fuchs_sondheimer_specular_t(delta, p):
    """The same S(delta, p) in the form usually quoted for films:
    1 - 3(1 - p)/(2 delta) int_1^inf (t^-3 - t^-5)(1 - e^{-delta t})/(1 - p e^{-delta t}) dt."""
    f = lambda t: (t ** -3 - t ** -5) * (-math.expm1(-delta * t)) / (1.0 - p * math.exp(-delta * t))
    val, _ = integrate.quad(f, 1.0, np.inf, limit=400, epsabs=1e-14)
    return 1.0 - 1.5 * (1.0 - p) / delta * val


def mode_table(mat):
    """(omega, v, tau, C) per mode from a workload material dict (numpy)."""
    T = mat["T_eq"]
    if mat["kind"] == "gray":
        return (np.zeros(1), np.array([mat["v"]]), np.array([mat["tau"]]), np.array([mat["C"]]))
    om, vs, ts, cs = [], [], [], []
    for br in mat["branches"]:
        c1, c2, g = br["c1"], br["c2"], br["degeneracy"]
        kmax = 2 * math.pi / mat["a_lattice"]
        if c2 < 0:
            kmax = min(kmax, c1 / (2 * abs(c2)))
        wmax = c1 * kmax + c2 * kmax ** 2
        nb = mat["n_bins"]
        dw = wmax / nb
        w = (np.arange(nb) + 0.5) * dw
        v = np.sqrt(c1 * c1 + 4 * c2 * w)
        k = 2 * w / (c1 + v)
        dos = k * k / (2 * math.pi ** 2 * v)
        x = HBAR * w / (KB * T)
        dfdT = x * np.exp(x) / (np.expm1(x) ** 2 * T)
        om.append(w)
        vs.append(v)
        cs.append(g * dos * HBAR * w * dfdT * dw)
        ts.append(1.0 / (mat["A"] * w ** 4 + mat["B"] * w * w * T * math.exp(-mat["C"] / T)))
    return tuple(np.concatenate(a) for a in (om, vs, ts, cs))


def kappa_bulk(mat):
    _, v, tau, C = mode_table(mat)
    return float(np.sum(C * v * v * tau) / 3.0)


def kappa_bulk_anisotropic(mat, g):
    """Bulk conductivity when a relaxation event turns the direction with
    mean cosine g about the incoming one (the mode is still redrawn from the
    normalised Eq. 2, independently of the direction).  A particle emitted by
    the gradient source in mode b with |cos| law about z contributes its first
    flight Lambda_b mu, and after its j-th relaxation a flight of mean length
    <Lambda>_s = sum_b (C_b/tau_b) Lambda_b / sum_b C_b/tau_b along a direction
    whose mean z-cosine is g^j mu, so
    kappa = 1/3 sum_b C_b v_b Lambda_b + 1/3 (sum_b C_b v_b) g <Lambda>_s / (1 - g),
    which is (1/3) C v Lambda / (1 - g) for a gray medium and the usual bulk
    value at g = 0."""
    _, v, tau, C = mode_table(mat)
    lam = v * tau
    lam_s = float(np.sum(C / tau * lam) / np.sum(C / tau))
    return float(np.sum(C * v * lam) / 3.0 + np.sum(C * v) / 3.0 * g * lam_s / (1.0 - g))


def kappa_film(mat, L, specularity=0.0):
    """In-plane film conductivity; walls diffuse, or specular with
    probability ``specularity`` (the same on both walls)."""
    _, v, tau, C = mode_table(mat)
    lam = v * tau
    if specularity == 0.0:
        S = fuchs_sondheimer(L / lam)
    else:
        S = np.array([fuchs_sondheimer_specular(d, specularity) for d in L / lam])
    return float(np.sum(C * v * v * tau / 3.0 * S))


# --------------------------------------------------------------------------
# Multi-mode slab between black walls: collision-density integral equation
# --------------------------------------------------------------------------
def slab_multimode_psi(Lambda, q_emit, p_scat, L, M=200, richardson=True):
    """Psi of a black-walled slab for a non-gray medium.

    Particles leave the hot wall with mode probabilities ``q_emit`` (the wall
    source weights C_b v_b) and a cosine law; every relaxation event redraws
    the mode with probabilities ``p_scat`` (normalised Eq. 2, C_b / tau_b) and
    an isotropic direction.  With equal and opposite wall excesses Psi equals
    the probability that a wall particle is absorbed by the opposite wall.

    The collision density F(x) obeys F = f0 + K F with
      f0(x)   = sum_b q_b (2/Lambda_b) E2(x/Lambda_b)         (first collisions)
      K(x,x') = sum_b p_b (1/(2 Lambda_b)) E1(|x-x'|/Lambda_b)  (isotropic re-emission)
    and Psi = sum_b q_b 2 E3(L/Lambda_b) + int F(x) sum_b p_b E2((L-x)/Lambda_b)/2 dx.
    Solved with piecewise-linear F (exact panel integrals), Richardson in M.
    This is a different formulation from ``slab_solution`` (collision density
    instead of emissive power), so for a gray medium the two cross-check."""
    Lam = np.asarray(Lambda, dtype=np.float64)
    q = np.asarray(q_emit, dtype=np.float64) / np.sum(q_emit)
    p = np.asarray(p_scat, dtype=np.float64) / np.sum(p_scat)

    def solve(Mn):
        h = L / Mn
        nodes = np.linspace(0.0, L, Mn + 1)
        K = np.zeros((Mn + 1, Mn + 1))
        for lam, pb in zip(Lam, p):
            if pb == 0.0:
                continue
            t = nodes / lam
            Wb = np.zeros_like(K)
            for j in range(Mn + 1):
                if j > 0:
                    a, b = t[j - 1], t[j]
                    Wb[:, j] += _lin_E1(a, b, -a / (b - a), 1.0 / (b - a), t)
                if j < Mn:
                    a, b = t[j], t[j + 1]
                    Wb[:, j] += _lin_E1(a, b, b / (b - a), -1.0 / (b - a), t)
            K += pb * 0.5 * Wb  # dx'/(2 Lambda) = dtau'/2
        f0 = np.zeros(Mn + 1)
        for lam, qb in zip(Lam, q):
            f0 += qb * 2.0 / lam * En(2, nodes / lam)
        F = np.linalg.solve(np.eye(Mn + 1) - K, f0)
        # escape-to-far-wall integral, exact per panel for linear F:
        # int_a^b F(x) E2((L-x)/lam)/2 dx, with s = (L-x)/lam
        psi = float(np.sum(q * 2.0 * En(3, L / Lam)))
        for lam, pb in zip(Lam, p):
            if pb == 0.0:
                continue
            acc = 0.0
            for j in range(Mn):
                xa, xb = nodes[j], nodes[j + 1]
                beta = (F[j + 1] - F[j]) / h
                alpha = F[j] - beta * xa
                sa, sb = (L - xa) / lam, (L - xb) / lam  # sa > sb
                # x = L - lam s, dx = -lam ds: int_{sb}^{sa} (alpha + beta (L - lam s)) E2(s) lam ds
                G0 = lambda s: -En(3, s)
                G1 = lambda s: -s * En(3, s) - En(4, s)
                acc += lam * ((alpha + beta * L) * (G0(sa) - G0(sb)) - beta * lam * (G1(sa) - G1(sb)))
            psi += pb * 0.5 * acc
        return psi

    p1 = solve(M)
    if not richardson:
        return p1
    p2 = solve(2 * M)
    return (4 * p2 - p1) / 3


def porous_first_flight_distance(L, pitch, radius, pos, omega):
    """Distance along unit directions ``omega`` (n x 3) from points ``pos``
    (n x 3, inside the solid of the unit cell) to the first boundary of the
    cell: the film faces x = 0, L, the unit-cell faces y, z = 0, pitch, or the
    cylindrical pore of the given radius along x through the cell centre.
    Written with numpy from the geometry alone (the ray-boundary algebra)."""
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    ox, oy, oz = omega[:, 0], omega[:, 1], omega[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        dx = np.where(ox > 0, (L - x) / ox, np.where(ox < 0, x / -ox, np.inf))
        dy = np.where(oy > 0, (pitch - y) / oy, np.where(oy < 0, y / -oy, np.inf))
        dz = np.where(oz > 0, (pitch - z) / oz, np.where(oz < 0, z / -oz, np.inf))
        d = np.minimum(dx, np.minimum(dy, dz))
        if radius > 0:
            ry, rz = y - 0.5 * pitch, z - 0.5 * pitch
            a = oy * oy + oz * oz
            b = ry * oy + rz * oz
            c = ry * ry + rz * rz - radius * radius
            disc = b * b - a * c
            t = (-b - np.sqrt(np.maximum(disc, 0.0))) / a  # nearer root; c > 0 outside the pore
            hit = (a > 0) & (disc >= 0) & (b < 0) & (t >= 0)
            d = np.where(hit, np.minimum(d, t), d)
    return d


def _first_flight_samples(L, pitch, radius, m, seed):
    """Scrambled Sobol points of the gradient source in a pored cell: positions
    uniform in the solid, directions with the |mu_z| law about z; returns
    |mu_z| and the distance to the first boundary of each."""
    from scipy.stats import qmc
    u = qmc.Sobol(d=5, scramble=True, seed=seed).random_base2(m)
    pos = np.column_stack([u[:, 0] * L, u[:, 1] * pitch, u[:, 2] * pitch])
    solid = (pos[:, 1] - 0.5 * pitch) ** 2 + (pos[:, 2] - 0.5 * pitch) ** 2 >= radius ** 2
    pos, u = pos[solid], u[solid]
    # |mu| law on [-1, 1] by inverting its CDF: |mu| = sqrt(|2w - 1|), sign of 2w - 1
    w = u[:, 3]
    mu = np.where(w < 0.5, -np.sqrt(np.abs(1.0 - 2.0 * w)), np.sqrt(np.abs(2.0 * w - 1.0)))
    phi = 2.0 * np.pi * u[:, 4]
    s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    omega = np.column_stack([s * np.cos(phi), s * np.sin(phi), mu])
    return np.abs(mu), porous_first_flight_distance(L, pitch, radius, pos, omega)


def kappa_first_event_porous(mat, L, pitch, radius, m=18, scrambles=4, chunk=4096):
    """Conductivity of a pored film (gradient along z) when every particle
    stops at its first event of any kind (relaxation, film face, pore or
    unit-cell face: ``max_events = 1``).

    A particle emitted in mode b, uniformly in the solid with the |mu_z| law
    about z and sign sgn(mu_z) (dT/dz < 0), contributes s L_z = |mu_z|
    min(l, d), l exponential of mean Lambda_b and d its distance to the first
    boundary; the mean over l is |mu_z| Lambda_b (1 - exp(-d / Lambda_b)).
    Modes are emitted with probability C_b v_b / sum C v, and the gradient
    source's normalisation gives kappa = (1/2) (solid fraction) sum_b C_b v_b
    E[|mu_z| Lambda_b (1 - exp(-d / Lambda_b))] (the bulk limit d -> inf is
    (1/3) sum C v Lambda).  The mean over positions and directions is taken
    by scrambled Sobol quasi-Monte Carlo (2^m points, positions in the pore
    rejected), independently scrambled ``scrambles`` times.  Returns (kappa,
    standard error of the scramble mean)."""
    _, v, tau, C = mode_table(mat)
    lam = v * tau
    frac = 1.0 - math.pi * radius * radius / (pitch * pitch)
    vals = []
    for r in range(scrambles):
        amu, d = _first_flight_samples(L, pitch, radius, m, 1206 + r)
        total = 0.0
        for i in range(0, lam.size, 64):
            lb = lam[i:i + 64]
            acc = np.zeros(lb.size)
            for j in range(0, d.size, chunk):
                dd, aa = d[j:j + chunk, None], amu[j:j + chunk, None]
                acc += np.sum(aa * lb[None, :] * -np.expm1(-dd / lb[None, :]), axis=0)
            total += float(np.sum(C[i:i + 64] * v[i:i + 64] * acc / d.size))
        vals.append(0.5 * frac * total)
    vals = np.array(vals)
    return float(vals.mean()), float(vals.std(ddof=1) / math.sqrt(len(vals))) if len(vals) > 1 else 0.0


def ballistic_slab_fractions(L, x_lo, x_hi, v, times, nx, n_mu=20000):
    """Free streaming between specular walls: particles start uniformly in
    x_lo < x < x_hi at t = 0 with isotropic directions (mu_x uniform on
    [-1, 1]) and speed v, never relax, and reflect specularly at x = 0 and
    x = L.  Returns the fraction of them in each of nx equal slabs of [0, L]
    at each time (array [len(times)][nx]).

    Mirror-unfolding the walls, a particle at x0 moving with mu sits at fold(x0
    + mu v t), fold the reflection of the line onto [0, L] (period 2L).  For a
    given displacement D the starting interval [x_lo + D, x_hi + D] is cut
    by the images 2nL + [a, b] and 2nL - [b, a] of slab [a, b]; the lengths of
    those pieces over x_hi - x_lo are the slab fractions, exact for each mu,
    and the midpoint rule over n_mu values of mu does the direction average
    (the integrand is continuous and piecewise smooth in mu)."""
    times = np.asarray(times, dtype=float)
    mu = (np.arange(n_mu) + 0.5) / n_mu * 2.0 - 1.0
    edges = np.linspace(0.0, L, nx + 1)
    out = np.zeros((times.size, nx))
    w = x_hi - x_lo
    for it, t in enumerate(times):
        D = mu * v * t
        lo, hi = x_lo + D, x_hi + D
        nmin = int(np.floor(lo.min() / (2 * L))) - 1
        nmax = int(np.ceil(hi.max() / (2 * L))) + 1
        for j in range(nx):
            a, b = edges[j], edges[j + 1]
            acc = np.zeros(n_mu)
            for n in range(nmin, nmax + 1):
                for ia, ib in ((2 * n * L + a, 2 * n * L + b), (2 * n * L - b, 2 * n * L - a)):
                    acc += np.clip(np.minimum(hi, ib) - np.maximum(lo, ia), 0.0, None)
            out[it, j] = float(np.mean(acc)) / w
    return out


def film_flux_profile(mat, L, n_bins, dTdz=-1.0e6, n_mu=400):
    """In-plane heat flux q_z of a film with diffuse walls, averaged over each
    of n_bins equal slabs in depth x, under a uniform dT/dz (the depth-resolved
    form of the Fuchs-Sondheimer solution).

    For mode b the flux density at depth x is its bulk value (1/3) C_b v_b
    Lambda_b |dT/dz| times 1 - (3/4) int_0^1 (1 - mu^2) [exp(-x / (Lambda_b
    mu)) + exp(-(L - x) / (Lambda_b mu))] dmu (the particles reaching x
    without relaxing since leaving a diffuse wall carry no flux); its depth
    mean is the Fuchs-Sondheimer factor S(L / Lambda_b).  The exponentials are
    averaged over each slab in closed form and the mu integral is taken by
    Gauss-Legendre quadrature."""
    _, v, tau, C = mode_table(mat)
    lam = v * tau
    x, w = np.polynomial.legendre.leggauss(n_mu)
    mu = 0.5 * (x + 1.0)
    wm = 0.5 * w
    edges = np.linspace(0.0, L, n_bins + 1)
    dx = L / n_bins
    out = np.zeros(n_bins)
    for i in range(0, lam.size, 256):
        lb = lam[i:i + 256, None, None]                 # modes
        m = mu[None, :, None]                           # directions
        a, b = edges[None, None, :-1], edges[None, None, 1:]
        lm = lb * m
        # slab means of exp(-x / lm) and exp(-(L - x) / lm)
        e1 = lm / dx * (np.exp(-a / lm) - np.exp(-b / lm))
        e2 = lm / dx * (np.exp(-(L - b) / lm) - np.exp(-(L - a) / lm))
        red = 0.75 * np.sum(wm[None, :, None] * (1.0 - m * m) * (e1 + e2), axis=1)   # [modes, bins]
        qb = (C[i:i + 256] * v[i:i + 256] * lam[i:i + 256] / 3.0)[:, None]
        out += np.sum(qb * (1.0 - red), axis=0)
    return out * abs(dTdz)


def porous_free_path_distance(L, pitch, radius, pos, omega, max_cells=64):
    """Distance along unit directions ``omega`` from points ``pos`` in the solid
    of the unit cell [0, L] x [0, pitch]^2 to the first film face (x = 0, L) or
    pore surface, the unit-cell faces being crossed freely (the periodic
    lattice of pores, one centred in every pitch x pitch cell).  A pore lies
    inside its cell (2 radius < pitch), so only the pores of the cells the
    ray's (y, z) projection passes through can be hit: those cells are walked
    in order (a 2-D cell walk), the first pore hit ending the walk.  Rays
    still running after ``max_cells`` cells (probability < 1e-8 here) keep
    their film-face distance.  Returns the distances and the number of rays
    cut short."""
    x, y, z = pos[:, 0], pos[:, 1], pos[:, 2]
    ox, oy, oz = omega[:, 0], omega[:, 1], omega[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        d = np.where(ox > 0, (L - x) / ox, np.where(ox < 0, x / -ox, np.inf))
        ci = np.floor(y / pitch)
        cj = np.floor(z / pitch)
        a = oy * oy + oz * oz
        active = a > 0
        t_in = np.zeros_like(d)
        for _ in range(max_cells):
            if not active.any():
                break
            # pore of the current cell: |(y, z) + t (oy, oz) - c| = radius
            ry = y - (ci + 0.5) * pitch
            rz = z - (cj + 0.5) * pitch
            b = ry * oy + rz * oz
            c = ry * ry + rz * rz - radius * radius
            disc = b * b - a * c
            t = (-b - np.sqrt(np.maximum(disc, 0.0))) / a
            hit = active & (disc >= 0) & (t >= 0) & (radius > 0)
            d = np.where(hit & (t < d), t, d)
            # leave the cell through the face ahead in y or z
            ty = np.where(oy > 0, ((ci + 1) * pitch - y) / oy, np.where(oy < 0, (ci * pitch - y) / oy, np.inf))
            tz = np.where(oz > 0, ((cj + 1) * pitch - z) / oz, np.where(oz < 0, (cj * pitch - z) / oz, np.inf))
            step_y = ty <= tz
            t_in = np.minimum(ty, tz)
            ci = np.where(step_y, ci + np.sign(oy), ci)
            cj = np.where(step_y, cj, cj + np.sign(oz))
            active = active & ~hit & (t_in < d)
    return d, int(np.sum(active))


def kappa_free_path_porous(mat, L, pitch, radius, m=17, scrambles=4, chunk=4096):
    """Conductivity of a pored film (gradient along z) when every particle
    stops at its first relaxation or film-face or pore hit, crossings of the
    periodic unit-cell faces not counted (``max_collisions = 1``): the
    ``kappa_first_event_porous`` construction with the distance to the first
    boundary taken through the periodic lattice of pores.  Returns (kappa,
    standard error of the scramble mean)."""
    from scipy.stats import qmc
    _, v, tau, C = mode_table(mat)
    lam = v * tau
    frac = 1.0 - math.pi * radius * radius / (pitch * pitch)
    vals = []
    for r in range(scrambles):
        u = qmc.Sobol(d=5, scramble=True, seed=1206 + r).random_base2(m)
        pos = np.column_stack([u[:, 0] * L, u[:, 1] * pitch, u[:, 2] * pitch])
        solid = (pos[:, 1] - 0.5 * pitch) ** 2 + (pos[:, 2] - 0.5 * pitch) ** 2 >= radius ** 2
        pos, u = pos[solid], u[solid]
        w = u[:, 3]
        mu = np.where(w < 0.5, -np.sqrt(np.abs(1.0 - 2.0 * w)), np.sqrt(np.abs(2.0 * w - 1.0)))
        phi = 2.0 * np.pi * u[:, 4]
        s = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
        omega = np.column_stack([s * np.cos(phi), s * np.sin(phi), mu])
        d, _ = porous_free_path_distance(L, pitch, radius, pos, omega)
        amu = np.abs(mu)
        total = 0.0
        for i in range(0, lam.size, 64):
            lb = lam[i:i + 64]
            acc = np.zeros(lb.size)
            for j in range(0, d.size, chunk):
                dd, aa = d[j:j + chunk, None], amu[j:j + chunk, None]
                acc += np.sum(aa * lb[None, :] * -np.expm1(-dd / lb[None, :]), axis=0)
            total += float(np.sum(C[i:i + 64] * v[i:i + 64] * acc / d.size))
        vals.append(0.5 * frac * total)
    vals = np.array(vals)
    return float(vals.mean()), float(vals.std(ddof=1) / math.sqrt(len(vals)))
