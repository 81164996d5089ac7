"""Seeded synthetic time-varying 2-D vector fields.

These stand in for the paper's datasets (Table I: SCF, CFVKV, HCBA, FS, DT),
which are not available: they reproduce shapes and value regimes only, not the
datasets' contents.  Every field is float32 with layout [T][H][W][2]
(interleaved u, v; j is the fast x axis, i the y axis).  x = column j, y = row
i; u is the x velocity, v the y velocity.  This module holds no arithmetic of
the compression method: it only draws inputs, shared by the oracle tests and
the GPU path.
"""
from __future__ import annotations

import os

import numpy as np

# workload name -> (H, W, T, relative error bound)
WORKLOADS = {
    "vortex64": (64, 64, 8, 1e-2),
    "street512": (512, 512, 100, 1e-3),
    "jets721": (721, 1440, 48, 1e-3),
    "turb1024": (1024, 1024, 200, 1e-3),
}


def _add_vortex(u, v, cx, cy, R, amp, sign, win=4.0):
    """Adds a Gaussian vortex with streamfunction psi = s*amp*R*exp(-r^2/(2R^2)),
    u = d(psi)/dy, v = -d(psi)/dx, evaluated in a +-win*R window."""
    H, W = u.shape
    r = int(np.ceil(win * R))
    i0, i1 = max(0, int(np.floor(cy)) - r), min(H, int(np.floor(cy)) + r + 2)
    j0, j1 = max(0, int(np.floor(cx)) - r), min(W, int(np.floor(cx)) + r + 2)
    if i0 >= i1 or j0 >= j1:
        return
    yy = np.arange(i0, i1, dtype=np.float64)[:, None] - cy
    xx = np.arange(j0, j1, dtype=np.float64)[None, :] - cx
    e = np.exp(-(xx * xx + yy * yy) / (2.0 * R * R))
    u[i0:i1, j0:j1] += -sign * amp * yy / R * e
    v[i0:i1, j0:j1] += sign * amp * xx / R * e


def vortex_sum(H=64, W=64, T=8, seed=1000, n_vortex=6, drift=0.5, noise=1e-3):
    """Sum of Gaussian vortices (random centres in [8, H-8]x[8, W-8], or the
    middle half of a smaller side, radii U[4,10], unit amplitude with random
    sign) whose centres drift `drift` cells per step in +x, plus N(0, noise)
    per component."""
    rng = np.random.default_rng(seed)
    mx, my = min(8.0, W / 4.0), min(8.0, H / 4.0)
    cx = rng.uniform(mx, W - mx, n_vortex)
    cy = rng.uniform(my, H - my, n_vortex)
    R = rng.uniform(4, 10, n_vortex)
    s = rng.choice([-1.0, 1.0], n_vortex)
    out = np.empty((T, H, W, 2), np.float32)
    for t in range(T):
        u = np.zeros((H, W))
        v = np.zeros((H, W))
        for k in range(n_vortex):
            _add_vortex(u, v, cx[k] + drift * t, cy[k], R[k], 1.0, s[k], win=6.0)
        u += rng.normal(0.0, noise, (H, W))
        v += rng.normal(0.0, noise, (H, W))
        out[t, :, :, 0] = u
        out[t, :, :, 1] = v
    return out


def vortex_street(H=512, W=512, T=100, seed=1001, period=10, speed=1.5, R=12.0, amp=1.0,
                  x0=64.0, offset=40.0, shear=0.3, noise=1e-3):
    """Von Karman-like street: vortex pairs at y = H/2 +- offset shed at x = x0
    every `period` steps with alternating sign, advected at `speed` cells per
    step in +x and dropped once past the domain; background shear
    u = shear*(i - H/2)/(H/2); plus N(0, noise)."""
    rng = np.random.default_rng(seed)
    out = np.empty((T, H, W, 2), np.float32)
    cy0 = H / 2.0
    first = -int(np.ceil((W - x0) / speed / period)) - 1
    for t in range(T):
        u = np.repeat((shear * (np.arange(H) - cy0) / cy0)[:, None], W, axis=1).astype(np.float64)
        v = np.zeros((H, W))
        for n in range(first, t // period + 1):
            ts = n * period
            if ts > t:
                continue
            x = x0 + speed * (t - ts)
            if x > W + 4 * R:
                continue
            sgn = 1.0 if n % 2 == 0 else -1.0
            _add_vortex(u, v, x, cy0 + offset, R, amp, sgn)
            _add_vortex(u, v, x, cy0 - offset, R, amp, -sgn)
        u += rng.normal(0.0, noise, (H, W))
        v += rng.normal(0.0, noise, (H, W))
        out[t, :, :, 0] = u
        out[t, :, :, 1] = v
    return out


def zonal_jets(H=721, W=1440, T=48, seed=1002, n_eddy=200, cell_m=27750.0, step_s=3600.0):
    """Wind-like lat-lon field in cells per step: zonal jets u = U(phi) sin(3 phi)
    with U ~ U[10,40] m/s per jet band, plus `n_eddy` Gaussian eddies (radius
    U[5,20] cells, amplitude U[5,30] m/s, random sign) moving with the local jet
    speed.  Row i is latitude 90 - 180 i/(H-1) degrees; no wrap in longitude."""
    rng = np.random.default_rng(seed)
    ms = step_s / cell_m  # m/s -> cells per step
    phi = np.deg2rad(90.0 - 180.0 * np.arange(H) / (H - 1))
    band = np.clip(np.floor((phi + np.pi / 2) / (np.pi / 3)).astype(int), 0, 5)
    U = rng.uniform(10, 40, 6)
    ujet = U[band] * np.sin(3 * phi) * ms
    cx = rng.uniform(0, W, n_eddy)
    cy = rng.uniform(20, H - 20, n_eddy)
    R = rng.uniform(5, 20, n_eddy)
    A = rng.uniform(5, 30, n_eddy) * ms
    s = rng.choice([-1.0, 1.0], n_eddy)
    vel = ujet[np.clip(np.round(cy).astype(int), 0, H - 1)]
    out = np.empty((T, H, W, 2), np.float32)
    for t in range(T):
        u = np.repeat(ujet[:, None], W, axis=1).astype(np.float64)
        v = np.zeros((H, W))
        for k in range(n_eddy):
            _add_vortex(u, v, cx[k] + vel[k] * t, cy[k], R[k], A[k], s[k])
        out[t, :, :, 0] = u
        out[t, :, :, 1] = v
    return out


def turbulence(H=1024, W=1024, T=200, seed=1004, k0=4.0, umax=1.5, substeps=2):
    """2-D decaying turbulence on a periodic H x W grid, in cells per step.
    Initial state: random phases, energy spectrum E(k) ~ k^-3 above the
    wavenumber k0 (cycles per domain) and rising as k^2 below it, velocity
    scaled to max |u| = umax.  The vorticity w is then carried by its
    own streamfunction (w = -lap psi, u = d psi / dy, v = -d psi / dx):
    pseudo-spectral, classical fourth-order Runge-Kutta (`substeps` per
    output step), 2/3 dealiasing and k^8 hyperviscosity; float32 FFTs."""
    import scipy.fft as sf
    workers = os.cpu_count() or 1
    rng = np.random.default_rng(seed)
    ky = (2 * np.pi * np.fft.fftfreq(H)).astype(np.float32)[:, None]
    kx = (2 * np.pi * np.fft.rfftfreq(W)).astype(np.float32)[None, :]
    k2 = ky * ky + kx * kx
    k2[0, 0] = 1.0
    # shell index in cycles per domain (square domain: H for rows)
    kc = np.sqrt((ky * H / (2 * np.pi)) ** 2 + (kx * W / (2 * np.pi)) ** 2)
    E = np.where(kc >= k0, np.maximum(kc, 1e-6) ** -3.0, (kc / k0) ** 2 * k0 ** -3.0)
    E[0, 0] = 0.0
    amp = np.sqrt(E / np.maximum(kc, 1e-6) ** 3).astype(np.float32)
    phase = rng.uniform(0, 2 * np.pi, amp.shape).astype(np.float32)
    psi_h = amp * np.exp(1j * phase).astype(np.complex64)
    w_h = (k2 * psi_h).astype(np.complex64)
    w_h[0, 0] = 0.0
    kmax = np.float32(2.0 / 3.0 * np.pi)
    dealias = ((np.abs(ky) < kmax) & (np.abs(kx) < kmax)).astype(np.float32)
    dt = np.float32(1.0 / substeps)
    nu = np.float32(1.0 / kmax ** 8)
    damp = np.exp(-nu * k2 ** 4 * dt).astype(np.float32)

    def velocity(wh):
        ph = wh / k2
        u = sf.irfft2(1j * ky * ph, s=(H, W), workers=workers)
        v = sf.irfft2(-1j * kx * ph, s=(H, W), workers=workers)
        return u, v

    def rhs(wh):
        u, v = velocity(wh)
        wx = sf.irfft2(1j * kx * wh, s=(H, W), workers=workers)
        wy = sf.irfft2(1j * ky * wh, s=(H, W), workers=workers)
        return -sf.rfft2(u * wx + v * wy, workers=workers) * dealias

    u, v = velocity(w_h)
    scale = np.float32(umax / max(np.abs(u).max(), np.abs(v).max()))
    w_h = (w_h * scale).astype(np.complex64)
    out = np.empty((T, H, W, 2), np.float32)
    for t in range(T):
        u, v = velocity(w_h)
        out[t, :, :, 0] = u
        out[t, :, :, 1] = v
        if t == T - 1:
            break
        for _ in range(substeps):  # classical Runge-Kutta, then the hyperviscous decay
            k1 = rhs(w_h)
            k2s = rhs(w_h + 0.5 * dt * k1)
            k3 = rhs(w_h + 0.5 * dt * k2s)
            k4 = rhs(w_h + dt * k3)
            w_h = ((w_h + dt / 6 * (k1 + 2 * k2s + 2 * k3 + k4)) * damp).astype(np.complex64)
    return out


def batch_specs(n=64, seed=2000):
    """The uneven batch: n vortex-sum fields, each side 128 * 2^U[0,3] cells
    rounded to a multiple of 16 (H and W drawn apart), T ~ U{10..200} steps,
    random drift U[0.2, 1.5] cells per step, one vortex per 2048 cells (at
    least 6), radii U[4, 10], random signs, N(0, 1e-3) noise; field f has
    seed `seed + 1 + f`.  Returns a list of dicts (H, W, T, seed, n_vortex,
    drift)."""
    rng = np.random.default_rng(seed)
    specs = []
    for f in range(n):
        H = max(16, int(round(128 * 2.0 ** rng.uniform(0, 3) / 16)) * 16)
        W = max(16, int(round(128 * 2.0 ** rng.uniform(0, 3) / 16)) * 16)
        T = int(rng.integers(10, 201))
        specs.append(dict(H=H, W=W, T=T, seed=seed + 1 + f, n_vortex=max(6, (H * W) // 2048),
                          drift=float(rng.uniform(0.2, 1.5))))
    return specs


def vortex_sum_device(H, W, T, seed, n_vortex, drift, noise=1e-3, device="cuda"):
    """The vortex-sum field of `vortex_sum` (same parameter draws, untruncated
    Gaussians) generated on a torch device: each vortex's streamfunction
    factors into a row and a column profile, so u and v of a slice are two
    [H, K] x [K, W] products; float64 profiles and products, float32 output;
    noise from a torch generator seeded with `seed`.  For inputs too large to
    draw quickly on the host."""
    import torch
    rng = np.random.default_rng(seed)
    mx, my = min(8.0, W / 4.0), min(8.0, H / 4.0)
    cx = rng.uniform(mx, W - mx, n_vortex)
    cy = rng.uniform(my, H - my, n_vortex)
    R = rng.uniform(4, 10, n_vortex)
    s = rng.choice([-1.0, 1.0], n_vortex)
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(int(seed))
    f64 = torch.float64
    i = torch.arange(H, dtype=f64, device=dev)[:, None]
    j = torch.arange(W, dtype=f64, device=dev)[None, :]
    Rt = torch.tensor(R, dtype=f64, device=dev)
    st = torch.tensor(s, dtype=f64, device=dev)
    yy = i - torch.tensor(cy, dtype=f64, device=dev)[None, :]       # [H, K]
    ey = torch.exp(-yy * yy / (2.0 * Rt * Rt))
    out = torch.empty((T, H, W, 2), dtype=torch.float32, device=dev)
    for t in range(T):
        xx = j.T - torch.tensor(cx + drift * t, dtype=f64, device=dev)[None, :]  # [W, K]
        ex = torch.exp(-xx * xx / (2.0 * Rt * Rt))
        # u = sum_k -s_k (y/R_k) e_k, v = sum_k s_k (x/R_k) e_k
        u = (-(st / Rt) * yy * ey) @ ex.T
        v = (st * ey) @ ((xx / Rt) * ex).T
        u += noise * torch.randn((H, W), generator=g, dtype=f64, device=dev)
        v += noise * torch.randn((H, W), generator=g, dtype=f64, device=dev)
        out[t, :, :, 0] = u.to(torch.float32)
        out[t, :, :, 1] = v.to(torch.float32)
    return out


def _cache_path(name):
    """File that holds a generated workload between processes: in the system's
    temporary directory (never inside the repository), named after the
    workload and a hash of this module's source, so that an edited generator
    never reads a stale field.  CPT_SYNTH_CACHE=0 turns the cache off."""
    import hashlib
    import tempfile
    if os.environ.get("CPT_SYNTH_CACHE", "1") == "0":
        return None
    with open(os.path.abspath(__file__), "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    return os.path.join(tempfile.gettempdir(), f"cpt_synth_{name}_{h}.npy")


def _cached(name, make):
    path = _cache_path(name)
    if path and os.path.exists(path):
        try:
            return np.load(path)
        except Exception:
            pass
    uv = make()
    if path:
        tmp = f"{path[:-4]}.{os.getpid()}.tmp.npy"
        try:
            np.save(tmp, uv)
            os.replace(tmp, path)
        except Exception:
            if os.path.exists(tmp):
                os.unlink(tmp)
    return uv


def workload(name):
    """Returns (uv, relative error bound) for a named workload.  The slow
    spectral turbulence field is generated once per machine and kept in a
    temporary file (see _cache_path)."""
    if name == "vortex64":
        return vortex_sum(64, 64, 8, seed=1000), 1e-2
    if name == "street512":
        return vortex_street(512, 512, 100, seed=1001), 1e-3
    if name == "jets721":
        return zonal_jets(721, 1440, 48, seed=1002), 1e-3
    if name == "turb1024":
        return _cached(name, lambda: turbulence(1024, 1024, 200, seed=1004)), 1e-3
    raise KeyError(name)


def linear_field(H, W, T, a, b, c, d, saddle=False):
    """u = x - (a + b t), v = +-(y - (c + d t)): one critical point per slice
    moving along a straight line (x = a + b t, y = c + d t)."""
    t = np.arange(T, dtype=np.float64)[:, None, None]
    y = np.arange(H, dtype=np.float64)[None, :, None]
    x = np.arange(W, dtype=np.float64)[None, None, :]
    u = x - (a + b * t) + 0 * y
    v = (y - (c + d * t)) + 0 * x
    if saddle:
        v = -v
    return np.stack([u, v], -1).astype(np.float32)


def centre_field(H, W, T, x0, y0):
    """u = -(y - y0), v = x - x0: a centre at (x0, y0) in every slice."""
    y = np.arange(H, dtype=np.float64)[None, :, None]
    x = np.arange(W, dtype=np.float64)[None, None, :]
    u = -(y - y0) + 0 * x + np.zeros((T, 1, 1))
    v = (x - x0) + 0 * y + np.zeros((T, 1, 1))
    return np.stack([u, v], -1).astype(np.float32)


def birth_field(H, W, T, x0, y0, k, t0):
    """u = (x - x0)^2 - k (t - t0), v = y - y0: no critical point before t0,
    two after (x = x0 +- sqrt(k (t - t0))), joined into one trajectory."""
    t = np.arange(T, dtype=np.float64)[:, None, None]
    y = np.arange(H, dtype=np.float64)[None, :, None]
    x = np.arange(W, dtype=np.float64)[None, None, :]
    u = (x - x0) ** 2 - k * (t - t0) + 0 * y
    v = (y - y0) + 0 * x + 0 * t
    return np.stack([u, v], -1).astype(np.float32)
