"""Seeded synthetic inputs for the 1D model problem (Sec. 4).

This module holds no arithmetic of the multigrid method: it only draws the
manufactured solution's coefficients and samples the right-hand side and the
exact solution at cell centres.  Both the CUDA path's tests and benchmark and
the CPU oracle's tests take their inputs from here.

Problem: -u'' = f on (0, 1), u(0) = u(1) = 0, N = 2^M cells, centres
x_i = (i + 1/2)/N.

* ``sine_series``: u = sum_{k=1..K} c_k sin(k pi x) with c_k ~ N(0,1)/k^2
  from ``numpy.random.default_rng(seed)``, so f = sum c_k (k pi)^2 sin(k pi x).
* ``paper_series``: the appendix program's problem, f = sum over odd j below
  N/16 of sin(j pi x)/j, u = sum sin(j pi x)/(j (j pi)^2).
* ``batch_sizes`` / ``sine_series_batch``: many independent problems (sizes
  2^m with m drawn uniformly; each problem a sine series with its own seed),
  generated on the device as one matrix product of the coefficients with the
  sampled sines.
* ``varcoef_series``: -(a u')' = f with a = exp(g/2) at the faces,
  g = amp * sum_{k=1..K} d_k cos(k pi x) (d_k ~ N(0,1)/k), the manufactured
  u = sine series, f = -(a u')' = -(a' u' + a u'') at the centres;
  ``varcoef_series_batch`` the same for many problems on the device.
* ``bratu_series``: the nonlinear problem -u'' + lam e^u = f with the
  manufactured solution u = scale * sum c_k sin(k pi x) (default scale 1/2),
  f = -u'' + lam e^u sampled at the centres.
"""
import numpy as np


def centres(M):
    n = 1 << M
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def sine_coefficients(nmodes, seed):
    """c_k = z_k / k^2 with z ~ N(0, 1) drawn from default_rng(seed), k = 1..nmodes."""
    rng = np.random.default_rng(seed)
    z = rng.standard_normal(nmodes)
    k = np.arange(1, nmodes + 1, dtype=np.float64)
    return z / k**2


def sine_series(M, nmodes, seed, scale=1.0):
    """(f, u_exact, c) sampled at the 2^M cell centres."""
    x = centres(M)
    c = scale * sine_coefficients(nmodes, seed)
    f = np.zeros_like(x)
    u = np.zeros_like(x)
    for k in range(1, nmodes + 1):
        s = np.sin(k * np.pi * x)
        f += c[k - 1] * (k * np.pi) ** 2 * s
        u += c[k - 1] * s
    return f, u, c


def batch_sizes(nprob, mmin, mmax, seed):
    """log2 sizes m ~ U{mmin .. mmax} of nprob problems (default_rng(seed))."""
    return np.random.default_rng(seed).integers(mmin, mmax + 1, size=nprob)


def sine_series_batch(M, seeds, nmodes, device):
    """(f, c): float64 tensor of len(seeds) * 2^M right-hand-side values on
    `device`, problem k holding sine_series(M, nmodes, seeds[k]), and the
    coefficient array (len(seeds), nmodes)."""
    import torch
    c = np.stack([sine_coefficients(nmodes, int(s)) for s in seeds])
    k = np.arange(1, nmodes + 1, dtype=np.float64)
    x = torch.from_numpy(centres(M)).to(device)
    kt = torch.from_numpy(k).to(device)
    S = torch.sin(torch.pi * kt[:, None] * x[None, :])                 # (nmodes, 2^M)
    cf = torch.from_numpy(c * (k * np.pi) ** 2).to(device)             # (B, nmodes)
    return (cf @ S).reshape(-1).contiguous(), c


def varcoef_series(M, nmodes, seed, amp=1.0, gmodes=16):
    """(f, u_exact, log_a) for -(a u')' = f: log_a at the 2^M + 1 faces
    x_j = j / 2^M, f and u_exact at the cell centres."""
    n = 1 << M
    d, c = _varcoef_coefficients(nmodes, seed, amp, gmodes)
    faces = np.arange(n + 1, dtype=np.float64) / n
    x = centres(M)
    log_a = np.zeros(n + 1)
    g = np.zeros_like(x)
    gp = np.zeros_like(x)
    for k in range(1, gmodes + 1):
        log_a += 0.5 * d[k - 1] * np.cos(k * np.pi * faces)
        g += 0.5 * d[k - 1] * np.cos(k * np.pi * x)
        gp -= 0.5 * d[k - 1] * k * np.pi * np.sin(k * np.pi * x)
    a = np.exp(g)
    ap = gp * a
    u = np.zeros_like(x)
    up = np.zeros_like(x)
    upp = np.zeros_like(x)
    for k in range(1, nmodes + 1):
        u += c[k - 1] * np.sin(k * np.pi * x)
        up += c[k - 1] * k * np.pi * np.cos(k * np.pi * x)
        upp -= c[k - 1] * (k * np.pi) ** 2 * np.sin(k * np.pi * x)
    f = -(ap * up + a * upp)
    return f, u, log_a


def _varcoef_coefficients(nmodes, seed, amp, gmodes):
    rng = np.random.default_rng(seed + 7919)
    d = amp * rng.standard_normal(gmodes) / np.arange(1, gmodes + 1)
    return d, sine_coefficients(nmodes, seed)


def varcoef_series_batch(M, seeds, nmodes, device, amp=1.0, gmodes=16, chunk=64):
    """(f, log_a): float64 tensors on `device` of len(seeds) problems of 2^M cells,
    problem k holding varcoef_series(M, nmodes, seeds[k]) (f at the centres,
    log_a at the 2^M + 1 faces), formed as matrix products of the coefficients
    with the sampled cosines and sines, `chunk` problems at a time."""
    import torch
    n = 1 << M
    kg = torch.arange(1, gmodes + 1, dtype=torch.float64, device=device)
    ku = torch.arange(1, nmodes + 1, dtype=torch.float64, device=device)
    x = torch.from_numpy(centres(M)).to(device)
    faces = torch.arange(n + 1, dtype=torch.float64, device=device) / n
    cos_f = torch.cos(torch.pi * kg[:, None] * faces[None, :])
    cos_g = torch.cos(torch.pi * kg[:, None] * x[None, :])
    sin_g = torch.sin(torch.pi * kg[:, None] * x[None, :])
    cos_u = torch.cos(torch.pi * ku[:, None] * x[None, :])
    sin_u = torch.sin(torch.pi * ku[:, None] * x[None, :])
    fs, las = [], []
    for c0 in range(0, len(seeds), chunk):
        co = [_varcoef_coefficients(nmodes, int(sd), amp, gmodes) for sd in seeds[c0:c0 + chunk]]
        d = torch.from_numpy(np.stack([e[0] for e in co])).to(device)
        c = torch.from_numpy(np.stack([e[1] for e in co])).to(device)
        las.append((0.5 * d) @ cos_f)
        g = (0.5 * d) @ cos_g
        gp = -(0.5 * d * kg * torch.pi) @ sin_g
        up = (c * ku * torch.pi) @ cos_u
        upp = -(c * (ku * torch.pi) ** 2) @ sin_u
        a = torch.exp(g)
        fs.append(-(gp * a * up + a * upp))
    return torch.cat(fs).reshape(-1).contiguous(), torch.cat(las).reshape(-1).contiguous()


def bratu_series(M, nmodes, seed, lam, scale=0.5):
    """(f, u_exact, c) for -u'' + lam e^u = f with u = scale * sine series."""
    x = centres(M)
    c = scale * sine_coefficients(nmodes, seed)
    f = np.zeros_like(x)
    u = np.zeros_like(x)
    for k in range(1, nmodes + 1):
        s = np.sin(k * np.pi * x)
        f += c[k - 1] * (k * np.pi) ** 2 * s
        u += c[k - 1] * s
    f += lam * np.exp(u)
    return f, u, c


def bratu_series_batch(M, seeds, nmodes, lam, device, scale=0.5):
    """float64 tensor of len(seeds) * 2^M right-hand-side values on `device`,
    problem k holding bratu_series(M, nmodes, seeds[k], lam, scale)[0]."""
    import torch
    c = scale * np.stack([sine_coefficients(nmodes, int(s)) for s in seeds])
    k = np.arange(1, nmodes + 1, dtype=np.float64)
    x = torch.from_numpy(centres(M)).to(device)
    kt = torch.from_numpy(k).to(device)
    S = torch.sin(torch.pi * kt[:, None] * x[None, :])                 # (nmodes, 2^M)
    u = torch.from_numpy(c).to(device) @ S                             # (B, 2^M)
    f = torch.from_numpy(c * (k * np.pi) ** 2).to(device) @ S + lam * torch.exp(u)
    return f.reshape(-1).contiguous()


def paper_series(M):
    """(f, u_exact): odd modes j < N/16 with f-amplitude 1/j (appendix program)."""
    n = 1 << M
    x = centres(M)
    f = np.zeros_like(x)
    u = np.zeros_like(x)
    for j in range(1, max(n // 16, 2), 2):
        s = np.sin(j * np.pi * x)
        f += s / j
        u += s / j / (j * np.pi) ** 2
    return f, u


def discrete_solution(M, c):
    """Exact solution of the discrete system for a sine-series right-hand side.

    The sampled sines are eigenvectors of the cell-centred operator with the
    odd-ghost wall (eigenvalue 4 n^2 sin^2(k pi / (2n))), so the discrete
    solution is the same series with each coefficient scaled by
    (k pi)^2 / lambda_k.  Used by the tests as a closed form.
    """
    n = 1 << M
    x = centres(M)
    u = np.zeros_like(x)
    for k in range(1, len(c) + 1):
        lam = 4.0 * n * n * np.sin(k * np.pi / (2 * n)) ** 2
        u += c[k - 1] * (k * np.pi) ** 2 / lam * np.sin(k * np.pi * x)
    return u
