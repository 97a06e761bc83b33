"""Per-component error scales of the DPR1 adjoint, for componentwise parity tests.

The adjoint of (lambda, V) with respect to (d, z, rho) sums one contribution per eigenpair k
(the implicit derivative of Eq. (Pick) and the explicit Eq. (Aeigenvec)).  With
s_j = d_j - lambda_k, v = x / ||x||, vbar = dL/dv_k, c = v . vbar, g = vbar - v c and p the index
of the largest |v_p|, both the oracle and the kernel evaluate it in the form that has no
cancellation at p (S2 = sum_{j != p} v_j^2, P = sum_{j != p} v_j vbar_j):
  g_p = vbar_p S2 - v_p P,  Lam = dL/dlambda_k + sum_{j != p} g_j v_j / s_j,  T_p = g_p v_p / s_p,
  lambdabar = Lam + T_p,
  dbar_j += lambdabar v_j^2 - g_j v_j / s_j  (j != p),   dbar_p += Lam v_p^2 - T_p S2,
  zbar_j += (g_j / s_j - 2 lambdabar v_j) / ||x||  (j != p),
  zbar_p += (g_p / s_p (S2 - v_p^2) - 2 Lam v_p) / ||x||,
  rhobar += lambdabar / (rho ||x||)^2.
A rounding error (or a relative perturbation of the pair (sigma, mu)) of size u in each
elementary quantity moves a component by at most a modest multiple of u times its scale: the
same expression with every quantity replaced by a bound of its magnitude and every difference
by a sum of magnitudes (a running error bound).  |g_j| is bounded by
G_j = |vbar_j| + |v_j| sum_i |v_i vbar_i| (j != p) and G_p = |vbar_p| S2 + |v_p| sum_{i != p} |v_i vbar_i|.
Where a component's scale is close to its value the component is well conditioned and must
agree to full relative accuracy; where the scale is much larger, the component is a
cancellation of larger contributions and agrees to u times its scale.
"""
import numpy as np


def adjoint_scales(d, z, rho, sigma, mu, grad_lam=None, grad_Vt=None):
    """(scale_d[n], scale_z[n], scale_rho) summed over the eigenpairs whose pairs (sigma, mu) are
    given (rows t of grad_lam and grad_Vt belong to pair t)."""
    d, z = np.asarray(d, dtype=np.float64), np.asarray(z, dtype=np.float64)
    sigma, mu = np.asarray(sigma, dtype=np.float64), np.asarray(mu, dtype=np.float64)
    m = sigma.size
    S = (d[None, :] - sigma[:, None]) - mu[:, None]
    X = z[None, :] / S
    mx = np.max(np.abs(X), axis=1, keepdims=True)
    xn = mx[:, 0] * np.sqrt(np.sum((X / mx) ** 2, axis=1))
    V = X / xn[:, None]
    del X
    aV, aS = np.abs(V), np.abs(S)
    rows = np.arange(m)
    p = np.argmax(aV, axis=1)
    isp = np.zeros(V.shape, dtype=bool)
    isp[rows, p] = True
    vp = aV[rows, p]
    S2 = np.sum(np.where(isp, 0.0, V * V), axis=1)
    if grad_Vt is not None:
        gV = np.asarray(grad_Vt, dtype=np.float64)
        aVG = np.abs(V * gV)
        A = np.sum(np.where(isp, 0.0, aVG), axis=1)
        G = np.abs(gV) + aV * (A + aVG[rows, p])[:, None]
        G[rows, p] = np.abs(gV[rows, p]) * S2 + vp * A
    else:
        G = np.zeros_like(V)
    T = G * aV / aS
    Ls = (np.abs(np.asarray(grad_lam, dtype=np.float64)) if grad_lam is not None else 0.0) + \
        np.sum(np.where(isp, 0.0, T), axis=1)
    Ts = T[rows, p]
    Lb = Ls + Ts
    cd = Lb[:, None] * V * V + T
    cd[rows, p] = Ls * vp * vp + Ts * S2
    cz = (G / aS + 2.0 * Lb[:, None] * aV) / xn[:, None]
    cz[rows, p] = (G[rows, p] / aS[rows, p] * (S2 + vp * vp) + 2.0 * Ls * vp) / xn
    return cd.sum(axis=0), cz.sum(axis=0), float(np.sum(Lb / (rho * xn) ** 2))


def componentwise(got, ref, scale, tau, well_conditioned=100.0, rel=1e-10):
    """Checks one gradient array component by component and returns a summary.

    Every component: |got - ref| <= tau * scale.  Components whose scale is at most
    `well_conditioned` times their magnitude (no cancellation worth the name) must also agree to
    `rel` relatively.  Returns dict(max_scaled, max_rel_well, n_well, n_total, ok)."""
    got, ref, scale = np.atleast_1d(got), np.atleast_1d(ref), np.atleast_1d(scale)
    err = np.abs(got - ref)
    scaled = err / np.maximum(scale, 1e-300)
    well = scale <= well_conditioned * np.abs(ref)
    relerr = err[well] / np.abs(ref[well])
    out = dict(max_scaled=float(scaled.max() / tau), max_rel_well=float(relerr.max()) if relerr.size else 0.0,
               n_well=int(well.sum()), n_total=int(ref.size),
               worst=int(np.argmax(scaled)))
    out["ok"] = bool(out["max_scaled"] <= 1.0 and out["max_rel_well"] <= rel)
    return out


def central_differences(loss, d, z, rho, rel=1e-4):
    """Per-coordinate central differences of loss(d, z, rho), Richardson-extrapolated from steps h
    and h/2 (h = rel times the distance from d_j to its nearest neighbour, rel |z_j|, rel rho)."""
    n = d.size
    gaps = np.abs(np.diff(d))

    def deriv(f, h):
        return (4.0 * (f(h / 2) - f(-h / 2)) / h - (f(h) - f(-h)) / (2 * h)) / 3.0

    gd, gz = np.empty(n), np.empty(n)
    for j in range(n):
        gap = min(gaps[j - 1] if j > 0 else np.inf, gaps[j] if j < n - 1 else np.inf)

        def fdj(h, j=j):
            x = d.copy()
            x[j] += h
            return loss(x, z, rho)

        def fzj(h, j=j):
            x = z.copy()
            x[j] += h
            return loss(d, x, rho)

        gd[j] = deriv(fdj, rel * gap)
        gz[j] = deriv(fzj, rel * abs(z[j]))
    gr = deriv(lambda h: loss(d, z, rho + h), rel * rho)
    return gd, gz, gr
