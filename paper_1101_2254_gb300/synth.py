"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path's tests and benchmark and by the
oracle's tests.  It holds none of the fitting method's arithmetic: it only
draws parameters, builds the PSF images that are *inputs* to the method, and
adds noise to an already rendered true image (which each caller renders with
its own implementation).

Parameter layout per component (the library's ABI):
    Sersic  (kind 1): x0, y0, I_e, r_e, n, q, pa_deg, c
    ExpDisk (kind 2): x0, y0, I_0, r_s, q, pa_deg, c
    Sky     (kind 3): s0
    Gaussian(kind 4): x0, y0, I_0, fwhm, q, pa_deg, c

Workloads (sizes and distributions as the galaxy-fitting configurations state
them; values the statement leaves open are marked "chosen"):
    stamp64   -- one 64x64 stamp, Sersic n=4 r_e=8 q=0.7 PA=30 at (32.3, 31.7),
                 I_e=1, sky 0.05, Gaussian PSF 25x25 FWHM 3, 5x5 oversampling in
                 the central 8x8, noise seed 0, guess perturbed 20 % (seed 1).
    stamp512  -- one 512x512 bulge (Sersic) + exponential disk + sky stamp,
                 Moffat PSF 65x65 beta 3 FWHM 4, 10x10 oversampling in the
                 central 20x20, 15 free parameters.
    batch4096 -- 4096 single-Sersic stamps, sides log-uniform in [32, 256],
                 per-stamp Moffat PSF 33x33 FWHM U[2, 5].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SERSIC, EXPDISK, SKY, GAUSSIAN, MOFFAT, KING, NUKER, PSF, SKYPLANE, SERSIC_F = range(1, 11)
NSLOTS = {SERSIC: 8, EXPDISK: 7, SKY: 1, GAUSSIAN: 7, MOFFAT: 8, KING: 9, NUKER: 10, PSF: 3,
          SKYPLANE: 3, SERSIC_F: 14}

SIGMA_READ = 0.01
GAIN = 1.0


# ------------------------------------------------------------------ PSFs
def _normalised_f32(img: np.ndarray) -> np.ndarray:
    img = img / img.sum()
    return img.astype(np.float32)


def gaussian_psf(size: int, fwhm: float) -> np.ndarray:
    """Circular Gaussian sampled at pixel centres, centre at (c, c), sum 1 (FP64) -> FP32."""
    assert size % 2 == 1
    c = (size - 1) // 2
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    y, x = np.mgrid[-c:c + 1, -c:c + 1].astype(np.float64)
    return _normalised_f32(np.exp(-(x * x + y * y) / (2.0 * s * s)))


def moffat_psf(size: int, fwhm: float, beta: float = 3.0) -> np.ndarray:
    """Moffat (1 + r^2/alpha^2)^-beta, alpha = FWHM / (2 sqrt(2^(1/beta) - 1))."""
    assert size % 2 == 1
    c = (size - 1) // 2
    alpha = fwhm / (2.0 * math.sqrt(2.0 ** (1.0 / beta) - 1.0))
    y, x = np.mgrid[-c:c + 1, -c:c + 1].astype(np.float64)
    return _normalised_f32((1.0 + (x * x + y * y) / (alpha * alpha)) ** (-beta))


def random_psf(size: int, seed: int) -> np.ndarray:
    """Asymmetric positive random kernel (pins the flip convention of the convolution)."""
    rng = np.random.default_rng(seed)
    return _normalised_f32(rng.uniform(0.05, 1.0, (size, size)))


# ----------------------------------------------------------------- noise
def add_noise(m_true: np.ndarray, seed: int, sigma_read: float = SIGMA_READ,
              gain: float = GAIN):
    """sigma^2 = sigma_read^2 + max(m_true, 0)/gain;  d = m_true + sigma * N(0, 1).

    The normal draws come from numpy's PCG64 ``default_rng(seed)`` in row-major
    order.  Returns (d, sigma) as float32.
    """
    m = np.asarray(m_true, np.float64)
    sigma = np.sqrt(sigma_read ** 2 + np.maximum(m, 0.0) / gain)
    z = np.random.default_rng(seed).standard_normal(m.shape)
    return (m + sigma * z).astype(np.float32), sigma.astype(np.float32)


def noise_sigma(m_true: np.ndarray, sigma_read: float = SIGMA_READ, gain: float = GAIN):
    m = np.asarray(m_true, np.float64)
    return np.sqrt(sigma_read ** 2 + np.maximum(m, 0.0) / gain).astype(np.float32)


# ------------------------------------------------------------ parameters
def slot_roles(kinds):
    """Role name per slot: pos, amp, rad, n, beta, q, pa, c, sky; King rt,
    kalpha; Nuker nalpha, nbeta, ngamma."""
    roles = []
    for k in kinds:
        if k == SERSIC:
            roles += ["pos", "pos", "amp", "rad", "n", "q", "pa", "c"]
        elif k == MOFFAT:
            roles += ["pos", "pos", "amp", "rad", "beta", "q", "pa", "c"]
        elif k in (EXPDISK, GAUSSIAN):
            roles += ["pos", "pos", "amp", "rad", "q", "pa", "c"]
        elif k == KING:
            roles += ["pos", "pos", "amp", "rad", "rt", "kalpha", "q", "pa", "c"]
        elif k == NUKER:
            roles += ["pos", "pos", "amp", "rad", "nalpha", "nbeta", "ngamma", "q", "pa", "c"]
        elif k == PSF:
            roles += ["pos", "pos", "amp"]
        elif k == SKY:
            roles += ["sky"]
        elif k == SKYPLANE:
            roles += ["sky", "skygx", "skygy"]
        elif k == SERSIC_F:
            roles += ["pos", "pos", "amp", "rad", "n", "q", "pa", "c",
                      "fa", "fphi", "fa", "fphi", "fa", "fphi"]
        else:
            raise ValueError(k)
    return roles


def perturb_guess(kinds, p_true, fixed, seed: int, frac: float = 0.2):
    """Each free slot p <- p (1 + frac u), u ~ U[-1, 1] from ``seed``; positions
    instead move by frac * r * u with r the owning component's radius.  The
    result is clipped into the default box (q <= 1, n in [0.2, 10], ...)."""
    p = np.array(p_true, np.float64, copy=True)
    roles = slot_roles(kinds)
    free = [i for i in range(len(p)) if not fixed[i]]
    u = np.random.default_rng(seed).uniform(-1.0, 1.0, len(free))
    off = 0
    radius_of = {}
    for k in kinds:
        ns = NSLOTS[k]
        for s in range(ns):
            radius_of[off + s] = p_true[off + 3] if k not in (SKY, SKYPLANE) else 1.0
        off += ns
    for ui, i in zip(u, free):
        if roles[i] == "pos":
            p[i] = p_true[i] + frac * radius_of[i] * ui
        else:
            p[i] = p_true[i] * (1.0 + frac * ui)
    for i, r in enumerate(roles):
        if r == "q":
            p[i] = min(max(p[i], 0.05), 1.0)
        elif r == "n":
            p[i] = min(max(p[i], 0.2), 10.0)
        elif r == "beta":
            p[i] = min(max(p[i], 0.5), 20.0)
        elif r == "rad":
            p[i] = max(p[i], 0.1)
        elif r == "pa":
            p[i] = p[i] % 180.0
        elif r == "c":
            p[i] = min(max(p[i], -1.9), 2.0)
        elif r == "rt":
            p[i] = max(p[i], 0.1)
        elif r in ("kalpha", "nalpha"):
            p[i] = min(max(p[i], 0.1), 10.0)
        elif r == "nbeta":
            p[i] = min(max(p[i], 0.0), 10.0)
        elif r == "ngamma":
            p[i] = min(max(p[i], 0.0), 2.0)
        elif r == "fa":
            p[i] = min(max(p[i], -0.3), 0.3)
    return p


def sersic_ie_for_flux(F, re, n, q):
    """I_e for total flux F (c = 0); library special functions only."""
    from scipy.special import gammaincinv, gammaln
    b = gammaincinv(2.0 * n, 0.5)
    return F / (2.0 * math.pi * q * re * re * n * math.exp(b + gammaln(2.0 * n) - 2.0 * n * math.log(b)))


@dataclass
class Stamp:
    """One fitting problem: everything but the rendered image."""
    H: int
    W: int
    kinds: list
    params: np.ndarray          # true parameters
    fixed: np.ndarray           # uint8 per slot
    psf: np.ndarray             # float32 P x P
    os_factor: int = 1
    os_box: int = 0
    noise_seed: int = 0
    guess_seed: int = 1
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def P(self):
        return self.psf.shape[0]

    @property
    def nslots(self):
        return len(self.params)

    @property
    def nfree(self):
        return int(len(self.fixed) - np.count_nonzero(self.fixed))

    def guess(self):
        return perturb_guess(self.kinds, self.params, self.fixed, self.guess_seed)


def stamp64() -> Stamp:
    kinds = [SERSIC, SKY]
    p = np.array([32.3, 31.7, 1.0, 8.0, 4.0, 0.7, 30.0, 0.0, 0.05])
    fixed = np.zeros(9, np.uint8)
    fixed[7] = 1  # boxiness held at 0: 8 free parameters
    return Stamp(64, 64, kinds, p, fixed, gaussian_psf(25, 3.0), os_factor=5, os_box=8,
                 noise_seed=0, guess_seed=1, name="stamp64")


def stamp512(seed: int = 11, size: int = 512, psf_size: int = 65, os_factor: int = 10,
             os_box: int = 20) -> Stamp:
    """Bulge + disk + sky; bulge I_e = 1, disk I_0 set by B/T ~ U[0.2, 0.8] (chosen)."""
    from scipy.special import gammaincinv, gammaln
    rng = np.random.default_rng(seed)
    ctr = size / 2.0 + rng.uniform(-2.0, 2.0, 2)
    n = rng.uniform(2.0, 6.0)
    re = rng.uniform(5.0, 30.0) * size / 512.0
    rs = rng.uniform(10.0, 60.0) * size / 512.0
    qb, qd = rng.uniform(0.3, 1.0, 2)
    pab, pad = rng.uniform(0.0, 180.0, 2)
    bt = rng.uniform(0.2, 0.8)
    b = gammaincinv(2.0 * n, 0.5)
    fb = 2.0 * math.pi * qb * re * re * n * math.exp(b + gammaln(2.0 * n) - 2.0 * n * math.log(b))
    fd = fb * (1.0 - bt) / bt
    i0 = fd / (2.0 * math.pi * qd * rs * rs)
    kinds = [SERSIC, EXPDISK, SKY]
    p = np.array([ctr[0], ctr[1], 1.0, re, n, qb, pab, 0.0,
                  ctr[0], ctr[1], i0, rs, qd, pad, 0.0,
                  0.05])
    fixed = np.zeros(16, np.uint8)
    fixed[14] = 1  # disk boxiness held: 15 free (bulge boxiness free)
    return Stamp(size, size, kinds, p, fixed, moffat_psf(psf_size, 4.0, 3.0),
                 os_factor=os_factor, os_box=os_box, noise_seed=0, guess_seed=1,
                 name=f"stamp{size}", extra=dict(bt=bt))


def batch_stamps(count: int = 4096, seed: int = 21, smin: int = 32, smax: int = 256,
                 psf_size: int = 33, noise_seed: int = 22):
    """Single-Sersic stamps: side log-uniform [smin, smax]; n ~ U[0.5, 6];
    r_e log-uniform [2, 40]; q ~ U[0.2, 1]; PA ~ U[0, 180); flux log-uniform
    [1e2, 1e5] (chosen); centre at the stamp centre +- U[-1, 1]; sky 0.05;
    Moffat PSF beta 3 with FWHM ~ U[2, 5]; 5x5 oversampling in the central 8x8
    (chosen).  Noise seeds are noise_seed * 1_000_003 + index."""
    rng = np.random.default_rng(seed)
    sides = np.exp(rng.uniform(math.log(smin), math.log(smax), count)).astype(np.int64)
    sides = np.clip(sides, smin, smax)
    out = []
    for i in range(count):
        s = int(sides[i])
        n = rng.uniform(0.5, 6.0)
        re = math.exp(rng.uniform(math.log(2.0), math.log(40.0)))
        q = rng.uniform(0.2, 1.0)
        pa = rng.uniform(0.0, 180.0)
        F = math.exp(rng.uniform(math.log(1e2), math.log(1e5)))
        ie = sersic_ie_for_flux(F, re, n, q)
        cx, cy = (s - 1) / 2.0 + rng.uniform(-1.0, 1.0, 2)
        fwhm = rng.uniform(2.0, 5.0)
        p = np.array([cx, cy, ie, re, n, q, pa, 0.0, 0.05])
        fixed = np.zeros(9, np.uint8)
        fixed[7] = 1
        out.append(Stamp(s, s, [SERSIC, SKY], p, fixed, moffat_psf(psf_size, fwhm, 3.0),
                         os_factor=5, os_box=min(8, s), noise_seed=noise_seed * 1_000_003 + i,
                         guess_seed=seed * 1_000_003 + i, name=f"batch[{i}]",
                         extra=dict(flux=F, fwhm=fwhm)))
    return out


def random_params(kinds, rng, H, W, n_range=(0.5, 6.0), boxy=False, beta_range=(1.5, 6.0)):
    """Random but well-inside-the-stamp parameters for parity tests."""
    p = []
    for k in kinds:
        if k == SKY:
            p += [rng.uniform(0.0, 0.1)]
            continue
        if k == SKYPLANE:
            p += [rng.uniform(0.0, 0.1), rng.uniform(-2e-3, 2e-3), rng.uniform(-2e-3, 2e-3)]
            continue
        x0 = rng.uniform(0.3 * W, 0.7 * W)
        y0 = rng.uniform(0.3 * H, 0.7 * H)
        amp = rng.uniform(0.5, 2.0)
        r = rng.uniform(2.0, 0.25 * min(H, W) + 2.0)
        q = rng.uniform(0.3, 1.0)
        pa = rng.uniform(0.0, 180.0)
        c = rng.uniform(-0.5, 0.5) if boxy else 0.0
        if k == SERSIC:
            p += [x0, y0, amp, r, rng.uniform(*n_range), q, pa, c]
        elif k == MOFFAT:
            p += [x0, y0, amp, r, rng.uniform(*beta_range), q, pa, c]
        elif k == KING:
            rc = rng.uniform(1.5, 0.1 * min(H, W) + 2.0)
            p += [x0, y0, amp, rc, rc * rng.uniform(4.0, 10.0), rng.uniform(1.5, 3.0), q, pa, c]
        elif k == NUKER:
            p += [x0, y0, amp, r, rng.uniform(1.0, 3.0), rng.uniform(2.5, 4.5),
                  rng.uniform(0.0, 0.8), q, pa, c]
        elif k == PSF:
            p += [x0, y0, rng.uniform(20.0, 100.0)]
        else:
            p += [x0, y0, amp, r, q, pa, c]
    return np.array(p, np.float64)


# ------------------------------------------------------ spectral lines, cubes
def gaussian_lsf(size: int, fwhm: float) -> np.ndarray:
    """Gaussian line-spread function sampled at channel offsets -c .. c, sum 1
    (FP64) -> FP32."""
    assert size % 2 == 1
    c = (size - 1) // 2
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    u = np.arange(-c, c + 1, dtype=np.float64)
    return _normalised_f32(np.exp(-u * u / (2.0 * s * s)))


def random_lsf(size: int, seed: int) -> np.ndarray:
    """Asymmetric positive random LSF (pins the flip of the convolution)."""
    return _normalised_f32(np.random.default_rng(seed).uniform(0.05, 1.0, size))


@dataclass
class SpecCube:
    """Spectra of a cube (one per spaxel) or any batch of spectra: everything
    but the rendered data.  params: count x (n_cont + 3 n_lines)."""
    n_chan: int
    n_lines: int
    n_cont: int
    params: np.ndarray
    lsf: np.ndarray              # float32 L (shared) or count x L
    noise_seed: int = 0
    guess_seed: int = 1
    name: str = ""

    @property
    def count(self) -> int:
        return self.params.shape[0]

    def guess(self, frac: float = 0.2) -> np.ndarray:
        """Each amplitude and width p <- p (1 + frac u), each centre moves by
        frac * width * u, the continuum a_j <- a_j (1 + frac u), u ~ U[-1, 1]
        from guess_seed; widths are kept at >= 0.25."""
        rng = np.random.default_rng(self.guess_seed)
        p = self.params.copy()
        u = rng.uniform(-1.0, 1.0, p.shape)
        nc = self.n_cont
        p[:, :nc] *= 1.0 + frac * u[:, :nc]
        for k in range(self.n_lines):
            a, m, s = nc + 3 * k, nc + 3 * k + 1, nc + 3 * k + 2
            p[:, a] *= 1.0 + frac * u[:, a]
            p[:, m] += frac * self.params[:, s] * u[:, m]
            p[:, s] = np.maximum(p[:, s] * (1.0 + frac * u[:, s]), 0.25)
        return p


def spec_batch(count: int, n_chan: int, n_lines: int, n_cont: int, lsf_size: int,
               seed: int, lsf_fwhm: float = 3.0, per_spectrum_lsf: bool = False,
               name: str = "") -> SpecCube:
    """Random spectra: a continuum of level U[20, 80] with a gentle slope and
    curvature, and lines of amplitude U[30, 300] (one in four absorbing, 0.4 to
    0.8 of the continuum deep), width U[1.5, 6] channels, centres spread over the
    middle 80 % of the band at least 4 widths apart."""
    rng = np.random.default_rng(seed)
    npar = n_cont + 3 * n_lines
    p = np.zeros((count, npar))
    cont = [lambda: rng.uniform(20.0, 80.0), lambda: rng.uniform(-5.0, 5.0),
            lambda: rng.uniform(-3.0, 3.0)]
    for b in range(count):
        for j in range(n_cont):
            p[b, j] = cont[j]()
        lo, hi = 0.1 * n_chan, 0.9 * n_chan
        slots = np.sort(rng.uniform(lo, hi, n_lines))
        for k in range(n_lines):
            s = rng.uniform(1.5, 6.0)
            A = rng.uniform(30.0, 300.0)
            if rng.uniform() < 0.25:
                A = -rng.uniform(0.4, 0.8) * (p[b, 0] if n_cont else 50.0)
            p[b, n_cont + 3 * k:n_cont + 3 * k + 3] = [A, slots[k], s]
        # separate the lines by at least 4 widths (shift the later ones)
        for k in range(1, n_lines):
            prev = p[b, n_cont + 3 * (k - 1) + 1] + 4.0 * max(p[b, n_cont + 3 * (k - 1) + 2],
                                                            p[b, n_cont + 3 * k + 2])
            p[b, n_cont + 3 * k + 1] = max(p[b, n_cont + 3 * k + 1], prev)
    if per_spectrum_lsf:
        lsf = np.stack([gaussian_lsf(lsf_size, rng.uniform(0.7, 1.3) * lsf_fwhm)
                        for _ in range(count)])
    else:
        lsf = gaussian_lsf(lsf_size, lsf_fwhm)
    return SpecCube(n_chan, n_lines, n_cont, p, lsf, noise_seed=seed * 7 + 1,
                    guess_seed=seed * 7 + 2, name=name or f"spec{count}x{n_chan}")


def spec_cube(side: int, n_chan: int, lsf_size: int = 25, seed: int = 0) -> SpecCube:
    """An integral-field cube of side x side spaxels (row-major), each spectrum
    an emission-line triplet like H-alpha with the [N II] doublet on a sloped
    continuum: fixed line spacing, a rotation-curve velocity field (centres
    shift by up to 6 % of the band across the disc), amplitudes falling off
    with radius, widths 2-4 channels."""
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:side, 0:side].astype(np.float64)
    xc = yc = (side - 1) / 2.0
    r = np.hypot(x - xc, y - yc) / max(side / 2.0, 1.0)
    phi = np.arctan2(y - yc, x - xc)
    v = 0.06 * n_chan * np.tanh(3.0 * r) * np.cos(phi)  # centre shift in channels
    base = 0.5 * n_chan + v
    sep = 0.03 * n_chan
    amp = 250.0 * np.exp(-1.5 * r) + 20.0
    p = np.zeros((side * side, 2 + 9))
    p[:, 0] = (40.0 + 10.0 * rng.uniform(-1, 1, side * side))
    p[:, 1] = rng.uniform(-3.0, 3.0, side * side)
    w = rng.uniform(2.0, 4.0, side * side)
    for k, (off, rel) in enumerate(((-sep, 0.35), (0.0, 1.0), (sep, 0.9))):
        p[:, 2 + 3 * k] = (amp * rel).ravel() * rng.uniform(0.9, 1.1, side * side)
        p[:, 3 + 3 * k] = (base + off).ravel()
        p[:, 4 + 3 * k] = w
    return SpecCube(n_chan, 3, 2, p, gaussian_lsf(lsf_size, 3.0), noise_seed=seed * 7 + 1,
                    guess_seed=seed * 7 + 2, name=f"cube{side}x{side}x{n_chan}")
