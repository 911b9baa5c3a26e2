"""FP64 CPU oracle for the Fresnel-scintillation hot path.

TEST INFRASTRUCTURE ONLY.  This module is a plain, slow, obviously correct
restatement of what the scintillation simulation of Habibi, Moniez, Ansari &
Rahvar ("Simulation of optical interstellar scintillation", A&A 2013,
arXiv:1301.0514) computes.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code,
table or constant generator with the CUDA library and imports nothing from it.

Every function states the passage of the paper it follows.  Arithmetic is
IEEE double precision throughout; the 2D FFT of scipy.fft (pocketfft, the same
library numpy's FFT is built on) serves as a library primitive through fft2 and
ifft2 below (its sign and scaling conventions are pinned against a direct DFT
and against the oracle's own radix-2 transform, fft_radix2, in the tests);
numpy's 1D real FFT serves the periodogram.
FFT_WORKERS sets how many host threads one transform may use (1 by default;
the full-size tests raise it to the host's core count).  Where the paper is silent or ambiguous the reading taken here is
named in the docstring ("Reading Rn").

Conventions used everywhere in this file
----------------------------------------
* Grid: N x N pixels of side ``pixel_km`` (Delta_1), L = N * Delta_1.
  Arrays are indexed ``[iy, ix]`` (row = y).
* Pixel centres sit at x_i = (i + 1/2) Delta_1 (Sect. 3.2.1, "pixel position
  centres").
* Frequencies: k_i = fftfreq(N, Delta_1) in cycles/km (FFT order).
* Forward transform carries exp(-2 pi i k x); the Fresnel transfer function is
  H(k) = exp(-i pi lambda z |k|^2) (Reading R6).
* Units: km for lengths, nm for wavelengths, pc for distances.

Parity status: every function is pinned by tests under ``tests/``
(test_oracle_*.py) except ``modulation_index`` for random screens, whose
statistical values in the paper are loose (parity unpinned for those values;
the function itself is pinned on closed-form maps).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace

import numpy as np
from scipy import fft as sfft
from scipy import special

KM_PER_PC = 3.0856775814913673e13
KM_PER_NM = 1.0e-12

# Philox4x32 round multipliers and Weyl key increments (Salmon, Moraes, Dror &
# Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11, Sect. 4).
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)

# Threads one 2D transform may use: a library setting that changes no arithmetic
# beyond the rounding order inside the transform.
FFT_WORKERS = 1


def fft2(x):
    """2D DFT over the last two axes, X_k = sum_j x_j exp(-2 pi i k.j / N) (no scaling)."""
    return sfft.fft2(x, workers=FFT_WORKERS)


def ifft2(x):
    """Inverse 2D DFT over the last two axes, with the + sign and the 1/N^2 factor."""
    return sfft.ifft2(x, workers=FFT_WORKERS)


@dataclass(frozen=True)
class ScreenParams:
    """Physical parameters of one screen and observation (units in field names)."""
    n: int
    pixel_km: float
    r_diff_km: float
    beta: float = 11.0 / 3.0
    lambda_nm: float = 500.0
    lambda_ref_nm: float = 500.0
    z_pc: float = 160.0
    source_radius_km: float = 0.0
    seed: int = 0
    screen_id: int = 0
    margin_km: float = -1.0   # <0: default min(10 R_F, L/4); 0: no taper

    def with_(self, **kw) -> "ScreenParams":
        return replace(self, **kw)


# ---------------------------------------------------------------------------
# Philox4x32-10 and Gaussian draws
# ---------------------------------------------------------------------------
def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Salmon et al. SC'11).

    Each round multiplies words 0 and 2 by the two round constants, crosses the
    high halves (xored with the other counter words and the key) into words
    0/2 and the low halves into words 1/3; the key is bumped by the Weyl
    constants between rounds.  Arguments are uint32-valued arrays (broadcast).
    Returns four uint64 arrays holding 32-bit words.
    """
    c = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3)]
    k = [np.asarray(x, dtype=np.uint64) & _MASK32 for x in (k0, k1)]
    for rnd in range(10):
        if rnd:
            k = [(k[0] + _PHILOX_W0) & _MASK32, (k[1] + _PHILOX_W1) & _MASK32]
        p0 = _PHILOX_M0 * c[0]
        p1 = _PHILOX_M1 * c[2]
        c = [((p1 >> np.uint64(32)) ^ c[1] ^ k[0]) & _MASK32,
             p1 & _MASK32,
             ((p0 >> np.uint64(32)) ^ c[3] ^ k[1]) & _MASK32,
             p0 & _MASK32]
    return c


def noise_words(n: int, seed: int, screen_id: int, rows=None):
    """Philox words for the spectral bins of one screen.

    Counter of bin (iy, ix) = (ix, iy, screen_id, 0); key = (seed low 32 bits,
    seed high 32 bits).  ``rows`` optionally restricts to a slice of iy.
    Returns four uint64 arrays of shape (len(rows), n).
    """
    iy = np.arange(n, dtype=np.uint64) if rows is None else np.asarray(rows, dtype=np.uint64)
    ix = np.arange(n, dtype=np.uint64)
    IY, IX = np.meshgrid(iy, ix, indexing="ij")
    seed = int(seed)
    return philox4x32_10(IX, IY, np.uint64(screen_id & 0xFFFFFFFF), np.uint64(0),
                         np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))


def uniform53(hi, lo):
    """Uniform in (0, 1): the top 53 bits of the 64-bit word (hi:lo), plus one half, times 2^-53."""
    w = (np.asarray(hi, dtype=np.uint64) << np.uint64(32)) | np.asarray(lo, dtype=np.uint64)
    return ((w >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def gaussian_pair(words):
    """Two independent standard normals per bin by the Box-Muller transform.

    u_a from words (w1:w0), u_b from words (w3:w2); r = sqrt(-2 ln u_a),
    g_re = r cos(2 pi u_b), g_im = r sin(2 pi u_b).
    """
    w0, w1, w2, w3 = words
    ua = uniform53(w1, w0)
    ub = uniform53(w3, w2)
    r = np.sqrt(-2.0 * np.log(ua))
    return r * np.cos(2.0 * np.pi * ub), r * np.sin(2.0 * np.pi * ub)


# ---------------------------------------------------------------------------
# Phase spectrum and screen synthesis (Sect. 2, Eq. spectre; Sect. 3.1, Eq. densite)
# ---------------------------------------------------------------------------
def f_beta(beta: float) -> float:
    """f(beta) = 2^-beta beta Gamma(-beta/2) / Gamma(beta/2) (Eq. spectre)."""
    return 2.0 ** (-beta) * beta * special.gamma(-beta / 2.0) / special.gamma(beta / 2.0)


def phase_spectrum(q, r_diff_km: float, beta: float):
    """S_phi(q) = R_diff^2 / (2 (2 pi)^(beta-1) f(beta)) * (R_diff q)^-beta (Eq. spectre).

    q in cycles/km; S in km^2 (so that Var(phi) = sum S dq^2).
    """
    q = np.asarray(q, dtype=np.float64)
    c = r_diff_km ** 2 / (2.0 * (2.0 * np.pi) ** (beta - 1.0) * f_beta(beta))
    with np.errstate(divide="ignore"):
        return c * (r_diff_km * q) ** (-beta)


def fft_freqs(n: int, pixel_km: float):
    """Spatial frequencies of the FFT bins, cycles/km, FFT order."""
    return np.fft.fftfreq(n, d=pixel_km)


def noise_spectrum(p: ScreenParams, rows=None):
    """Random phase spectrum F_phi of Eq. densite.

    F = (f_re + i f_im)/sqrt(2) with f ~ N(0, L_x L_y S_phi(q)) as a *variance*
    (Reading R1: this is what makes <|F|^2> = L_x L_y S).  The DC bin, where S
    diverges, is set to zero; every other FFT bin is kept, Nyquist row and
    column included, with the square cutoff of the grid (Reading R4).
    """
    n = p.n
    L = n * p.pixel_km
    k = fft_freqs(n, p.pixel_km)
    ky = k if rows is None else k[np.asarray(rows)]
    Q = np.sqrt(ky[:, None] ** 2 + k[None, :] ** 2)
    S = phase_spectrum(Q, p.r_diff_km, p.beta)
    S[Q == 0.0] = 0.0                         # DC bin: F = 0
    sigma = np.sqrt(L * L * S)
    g_re, g_im = gaussian_pair(noise_words(n, p.seed, p.screen_id, rows))
    return sigma * (g_re + 1j * g_im) / np.sqrt(2.0)


def make_screen(p: ScreenParams):
    """Phase screen phi(x_1, y_1) in radians, at lambda_ref (Sect. 3.1).

    phi_j = sqrt(2)/(L_x L_y) * Re sum_k F_k exp(+2 pi i k . x_j): the inverse
    Fourier transform with measure dq = 1/L, keeping sqrt(2) times the real part
    so that phi has covariance sum_k S_k dq^2 cos(2 pi k . r) (Reading R2).
    """
    n = p.n
    L = n * p.pixel_km
    # the spectrum bin by bin, drawn a few rows at a time (each bin's draw depends on
    # its own counter only, so the rows can be taken in any grouping)
    step = max(1, (1 << 16) // n)
    F = np.concatenate([noise_spectrum(p, rows=np.arange(r, min(r + step, n))) for r in range(0, n, step)])
    # ifft2 divides by N^2; multiply it back to get the plain sum.
    return np.sqrt(2.0) / (L * L) * np.real(ifft2(F)) * (n * n)


def structure_function_discrete(n: int, pixel_km: float, r_diff_km: float, beta: float, r_km):
    """Expected structure function of the sampled screen along x.

    E[D(r)] = 2 sum_k S(q_k) dq^2 (1 - cos(2 pi k_x r)) over every FFT bin but
    DC: the spectrum "sampled as in the simulation" of Sect. 3.1.1 (Eq. crec with
    the sampled theoretical spectrum).
    """
    k = fft_freqs(n, pixel_km)
    dq = 1.0 / (n * pixel_km)
    r_km = np.atleast_1d(np.asarray(r_km, dtype=np.float64))
    k2y = k ** 2
    acc = np.zeros_like(r_km)
    for j0 in range(0, n, 512):
        kx = k[j0:j0 + 512]
        Q = np.sqrt(k2y[:, None] + kx[None, :] ** 2)
        S = phase_spectrum(Q, r_diff_km, beta)
        if j0 == 0:
            S[0, 0] = 0.0
        Sx = S.sum(axis=0)                      # sum over k_y for each k_x
        acc += (Sx[None, :] * (1.0 - np.cos(2.0 * np.pi * kx[None, :] * r_km[:, None]))).sum(axis=1)
    return 2.0 * dq * dq * acc


# ---------------------------------------------------------------------------
# Screen check of Sect. 3.1.1: spectrum and structure function recomputed from
# the generated F_phi (Eq. crec), and R_diff^rec from D_rec(R_diff^rec) = 1.
# ---------------------------------------------------------------------------
def annulus_index(mx, my):
    """Annulus of the integer wave vector (mx, my): the nearest integer to |m|.

    The paper averages |F|^2 over the circle of radius q without a bin width;
    here (Reading R15) annulus j collects the FFT bins with j - 1/2 <= |m| < j + 1/2,
    i.e. width dq = 1/L centred on q_j = j/L.  |m| is never a half-integer for
    integer mx, my, so the assignment is unambiguous.
    """
    mx = np.asarray(mx, dtype=np.int64)
    my = np.asarray(my, dtype=np.int64)
    return np.floor(np.sqrt((mx * mx + my * my).astype(np.float64)) + 0.5).astype(np.int64)


def max_annulus(n: int) -> int:
    """Largest annulus index of an n x n grid (its corner, |m| = sqrt(2) n/2)."""
    return int(annulus_index(n // 2, n // 2))


def spectrum_rec(p: ScreenParams, j_max=None):
    """S_rec(q_j) = <|F_phi|^2>_{annulus j} / (L_x L_y) for j = 0..j_max (Sect. 3.1.1),
    from the generated F_phi of noise_spectrum, and the number of bins per annulus.

    Only spectral rows with |m_y| <= j_max can reach annuli j <= j_max, so a
    small j_max touches few rows.  Annuli without bins get S_rec = 0.
    """
    n = p.n
    L = n * p.pixel_km
    top = max_annulus(n)
    j_max = top if j_max is None else min(int(j_max), top)
    m = np.rint(np.fft.fftfreq(n) * n).astype(np.int64)          # signed integer frequencies
    rows = np.nonzero(np.abs(m) <= j_max)[0]
    F = noise_spectrum(p, rows)
    j = annulus_index(m[None, :], m[rows][:, None])
    keep = j <= j_max
    power = np.abs(F[keep]) ** 2
    sums = np.bincount(j[keep], weights=power, minlength=j_max + 1)
    counts = np.bincount(j[keep], minlength=j_max + 1)
    s = np.zeros(j_max + 1)
    nz = counts > 0
    s[nz] = sums[nz] / counts[nz] / (L * L)
    return s, counts


def structure_function_rec(s_rec, n: int, pixel_km: float, r_km):
    """D_rec(r) = 2 (xi_rec(0) - xi_rec(r)) with Eq. crec,
        xi_rec(r) = int_{q_min}^{q_max} 2 pi q S_rec(q) J0(2 pi q r) dq,
    evaluated on the annuli: q_j = j dq, dq = 1/L, j = 1..J with q_min = 1/L and
    q_max = 1/(2 Delta_1), the paper's 1D limits (J = n/2, or fewer if s_rec is
    shorter), each annulus weighted by its width dq (midpoint rule, Reading R15).
    """
    s_rec = np.asarray(s_rec, dtype=np.float64)
    L = n * pixel_km
    dq = 1.0 / L
    J = min(len(s_rec) - 1, n // 2)
    q = np.arange(1, J + 1) * dq
    S = s_rec[1:J + 1]
    r = np.atleast_1d(np.asarray(r_km, dtype=np.float64))
    arg = 2.0 * np.pi * q[None, :] * r[:, None]
    return 2.0 * (2.0 * np.pi * q[None, :] * S[None, :] * (1.0 - special.j0(arg))).sum(axis=1) * dq


def rdiff_rec(s_rec, n: int, pixel_km: float, iterations: int = 64) -> float:
    """R_diff^rec: the root of D_rec(R) = 1 on (0, L/2], by bisection from that
    bracket (nan when D_rec(L/2) < 1, i.e. the screen never decorrelates by 1 rad^2)."""
    lo, hi = 0.0, 0.5 * n * pixel_km
    if structure_function_rec(s_rec, n, pixel_km, hi)[0] < 1.0:
        return float("nan")
    for _ in range(iterations):
        mid = 0.5 * (lo + hi)
        if structure_function_rec(s_rec, n, pixel_km, mid)[0] < 1.0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# ---------------------------------------------------------------------------
# Illumination pattern (Sect. 2 Eq. hxy, Sect. 3.2)
# ---------------------------------------------------------------------------
def fresnel_radius_km(lambda_nm: float, z_pc: float) -> float:
    """R_F = sqrt(lambda z_0 / 2 pi) (Eq. hxy, Eq. Rfresnel)."""
    return math.sqrt(lambda_nm * KM_PER_NM * z_pc * KM_PER_PC / (2.0 * math.pi))


def aliasing_onset_px(fresnel_radius_km_: float, pixel_km: float) -> float:
    """Distance from the optical axis, in pixels, beyond which the quadratic phase
    exp(i x^2 / 2 R_F^2) is undersampled: x/Delta > pi (R_F/Delta)^2 - 1 (Eq. alias1)."""
    return math.pi * (fresnel_radius_km_ / pixel_km) ** 2 - 1.0


def taper_margin_km(p: ScreenParams, lambda_nm: float) -> float:
    """Taper margin L_m (Sect. 3.2.1): 10 R_F, clamped to L/4 so that two margins fit (Reading R3)."""
    if p.margin_km >= 0.0:
        return float(p.margin_km)
    L = p.n * p.pixel_km
    return min(10.0 * fresnel_radius_km(lambda_nm, p.z_pc), L / 4.0)


def taper_1d(n: int, pixel_km: float, margin_km: float):
    """Smoothing function SF(x) of Sect. 3.2.1 at the pixel centres x_i = (i+1/2) Delta.

    Raised sine over the margin L_m on each side, 1 in between; margin 0 gives 1.
    """
    x = (np.arange(n) + 0.5) * pixel_km
    if margin_km <= 0.0:
        return np.ones(n)
    L = n * pixel_km
    Lm = margin_km
    sf = np.ones(n)
    lo = x <= Lm
    hi = x >= L - Lm
    sf[lo] = 0.5 * (1.0 + np.sin(np.pi * x[lo] / Lm - np.pi / 2.0))
    sf[hi] = 0.5 * (1.0 + np.sin(np.pi * (x[hi] - L + Lm) / Lm + np.pi / 2.0))
    return sf


def fft_radix2(x, inverse: bool = False):
    """DFT of every line along the last axis by the iterative radix-2 Cooley-Tukey algorithm.

    N must be a power of two.  The input is put in bit-reversed order, then log2 N
    butterfly stages combine blocks of 2h elements: for k < h,
    X_k = a_k + w^k b_k and X_{k+h} = a_k - w^k b_k with w = exp(-+ 2 pi i / (2h)).
    Forward: X_k = sum_j x_j exp(-2 pi i j k / N); inverse: the + sign, no 1/N.
    The oracle's steps use scipy's FFT (fft2, ifft2) as their library primitive;
    this is the oracle's own transform, against which that primitive is pinned
    (with the direct DFT) in the tests.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    if n < 1 or n & (n - 1):
        raise ValueError("length must be a power of two")
    bits = n.bit_length() - 1
    j = np.arange(n)
    rev = np.zeros(n, dtype=np.int64)
    for b in range(bits):
        rev |= ((j >> b) & 1) << (bits - 1 - b)
    y = x[..., rev]
    sign = 1.0 if inverse else -1.0
    h = 1
    while h < n:
        w = np.exp(sign * 1j * np.pi * np.arange(h) / h)
        blocks = y.reshape(x.shape[:-1] + (n // (2 * h), 2, h))
        a = blocks[..., 0, :]
        b = blocks[..., 1, :] * w
        y = np.stack([a + b, a - b], axis=-2).reshape(x.shape)
        h *= 2
    return y


def fft2_radix2(x, inverse: bool = False):
    """2D DFT (both axes) by fft_radix2: lines along x, then along y."""
    y = fft_radix2(x, inverse)
    return np.swapaxes(fft_radix2(np.swapaxes(y, -1, -2), inverse), -1, -2)


def transfer_function(n: int, pixel_km: float, lambda_nm: float, z_pc: float):
    """Fresnel transfer function H(k) = exp(-i pi lambda z (k_x^2 + k_y^2)) (Reading R6).

    The exponential of the sum is the product h(k_y) h(k_x) of the 1D factors
    h(k) = exp(-i pi lambda z k^2) = cos(pi lambda z k^2) - i sin(pi lambda z k^2).
    """
    k = fft_freqs(n, pixel_km)
    lz = lambda_nm * KM_PER_NM * z_pc * KM_PER_PC
    theta = np.pi * lz * k ** 2
    h = np.cos(theta) - 1j * np.sin(theta)
    return h[:, None] * h[None, :]


def screen_field(phi, p: ScreenParams, lambda_nm: float):
    """Field behind the screen, A_in = SF(x) SF(y) exp(i phi lambda_ref / lambda).

    The phase of a fixed column density scales as 1/lambda (Eq. phiNl,
    Sect. 3.2.4); the taper multiplies the complex amplitude (Reading R3).
    """
    s = p.lambda_ref_nm / lambda_nm
    sf = taper_1d(p.n, p.pixel_km, taper_margin_km(p, lambda_nm))
    t = phi * s
    return (sf[:, None] * sf[None, :]) * (np.cos(t) + 1j * np.sin(t))


def propagate_field(a_in, pixel_km: float, lambda_nm: float, z_pc: float):
    """A_out = IDFT(DFT(A_in) H): exact Fresnel propagation of the periodic screen (Eq. hxy)."""
    H = transfer_function(a_in.shape[0], pixel_km, lambda_nm, z_pc)
    return ifft2(fft2(a_in) * H)


def fresnel_direct(a_in, pixel_km: float, lambda_nm: float, z_pc: float):
    """Direct Fresnel-Huygens sum over the screen pixels (Eq. hxy, discretised).

    A_out(x_0) = sum_{x_1} Delta^2/(i lambda z) exp(i pi |x_0 - x_1|^2 / (lambda z)) A_in(x_1),
    with the plain (non-periodic) pixel offsets.  O(N^4): tiny grids only.
    Note exp(i |d|^2 / 2R_F^2) = exp(i pi |d|^2 / lambda z).
    """
    n = a_in.shape[0]
    lz = lambda_nm * KM_PER_NM * z_pc * KM_PER_PC
    idx = np.arange(n)
    d = (idx[:, None] - idx[None, :]) * pixel_km          # d[o, i] = x_o - x_i
    kern1 = np.exp(1j * np.pi * d * d / lz)               # separable factor
    pref = pixel_km * pixel_km / (1j * lz)
    # A_out[oy, ox] = pref * sum_{iy, ix} k[oy, iy] k[ox, ix] A[iy, ix]
    return pref * (kern1 @ a_in @ kern1.T)


def intensity_mono(phi, p: ScreenParams, lambda_nm: float | None = None):
    """Point-source intensity h = |A_out|^2 at one wavelength (Eq. hxy).

    h is normalised to the intensity of an unobstructed plane wave (the
    1/(2 pi R_F^2) prefactor of Eq. hxy, inside the modulus): a uniform screen
    without taper gives exactly 1, and with the taper it stays 1 inside the
    fiducial zone (the uniformity check of Sect. 3.2.1).  Reading R5.
    """
    lam = p.lambda_nm if lambda_nm is None else lambda_nm
    a_in = screen_field(phi, p, lam)
    a_out = propagate_field(a_in, p.pixel_km, lam, p.z_pc)
    return np.abs(a_out) ** 2


def observer_pixel_km(p: ScreenParams, lambda_nm: float) -> float:
    """Pixel of the observer-plane pattern of the one-FFT method: Delta_0 = lambda z / (N Delta_1)
    (the conjugate variable of Eq. intens sampled by an N-point transform; Delta_0 = Delta_1 is the
    paper's N Delta_1^2 = 2 pi R_F^2 of Sect. 3.2.5)."""
    return lambda_nm * KM_PER_NM * p.z_pc * KM_PER_PC / (p.n * p.pixel_km)


def propagate_conjugate(phi, p: ScreenParams, lambda_nm: float | None = None):
    """Point-source pattern by the paper's one-FFT method (Eq. intens with Eq. Gxy):

        h(x_0) = |FT[SF(x_1) SF(y_1) G](x_0 / (lambda z))|^2 / (lambda z)^2,
        G = exp(i (phi lambda_ref/lambda + |x_1|^2 / (2 R_F^2))),

    the 1/(2 pi R_F^2) prefactor inside the modulus as in Reading R5 (a uniform screen gives 1).
    Coordinates take integer multiples of the pixel about the optical axis (Sect. 3.2.1, Reading
    R16): x_1 = (i - N/2) Delta_1 on the screen and x_0 = (k - N/2) Delta_0 on the observer
    plane, Delta_0 = lambda z / (N Delta_1); the taper uses the same pixels, at (i + 1/2) Delta_1
    from the screen edge.  The Fourier integral is the plain sum over pixels,
        FT[G](x_0 / lambda z) = Delta_1^2 sum_i G_i exp(-2 pi i x_1 . x_0 / (lambda z)),
    whose kernel is exp(-2 pi i (i - N/2)(k - N/2) / N): the DFT with both indices shifted by
    N/2 (numpy's fftshift(fft2(ifftshift(.)))).
    """
    lam = p.lambda_nm if lambda_nm is None else lambda_nm
    n = p.n
    lz = lam * KM_PER_NM * p.z_pc * KM_PER_PC
    x1 = (np.arange(n) - n // 2) * p.pixel_km
    a_in = screen_field(phi, p, lam)
    g = a_in * np.exp(1j * np.pi * (x1[:, None] ** 2 + x1[None, :] ** 2) / lz)
    ft = np.fft.fftshift(fft2(np.fft.ifftshift(g))) * p.pixel_km ** 2
    return np.abs(ft) ** 2 / lz ** 2


def sum_passband_conjugate(phi, p: ScreenParams, lambdas_nm, weights=None):
    """Passband co-addition (Sect. 3.2.4) of one-FFT patterns, whose pixels differ per
    wavelength (Delta_0 proportional to lambda).  Every pattern is resampled onto the grid of
    p.lambda_nm about the optical axis, which is a pixel centre of every grid (Sect. 3.2.1 puts
    pixel centres at integers so that patterns of different pixel sizes combine simply): output
    pixel k samples pattern l at u = (k - N/2) lambda_grid/lambda_l + N/2
    (pattern pixels), bilinearly, periodic like the discrete transform (Reading R16).
    """
    lambdas_nm = np.asarray(lambdas_nm, dtype=np.float64)
    w = np.full(len(lambdas_nm), 1.0 / len(lambdas_nm)) if weights is None else np.asarray(weights, float)
    n = p.n
    k = np.arange(n, dtype=np.float64) - n // 2
    out = np.zeros((n, n))
    for lam, wl in zip(lambdas_nm, w):
        h = propagate_conjugate(phi, p, lam)
        r = p.lambda_nm / lam
        u = k * r + n // 2
        X, Y = np.meshgrid(u, u)                       # X[row, col] = u[col], Y[row, col] = u[row]
        out += wl * bilinear_periodic(h, X.ravel(), Y.ravel()).reshape(n, n)
    return out


def sum_passband(phi, p: ScreenParams, lambdas_nm, weights=None):
    """Passband co-addition (Sect. 3.2.4): sum_l w_l I_l with sum w = 1 (flat 1/N_l by default)."""
    lambdas_nm = np.asarray(lambdas_nm, dtype=np.float64)
    if weights is None:
        weights = np.full(lambdas_nm.shape, 1.0 / lambdas_nm.size)
    out = np.zeros((p.n, p.n))
    for lam, w in zip(lambdas_nm, np.asarray(weights, dtype=np.float64)):
        out += w * intensity_mono(phi, p, lam)
    return out


# ---------------------------------------------------------------------------
# Extended source (Sect. 3.2.3, Eq. iprh)
# ---------------------------------------------------------------------------
def source_kernel(n: int, pixel_km: float, radius_km: float):
    """Fourier transform of the unit-integral uniform disk of radius R_s (Eq. iprh).

    K(q) = 2 J_1(2 pi q R_s) / (2 pi q R_s), K(0) = 1 (Reading R9).
    """
    k = fft_freqs(n, pixel_km)
    Q = np.sqrt(k[:, None] ** 2 + k[None, :] ** 2)
    if radius_km <= 0.0:
        return np.ones((n, n))
    x = 2.0 * np.pi * Q * radius_km
    K = np.ones_like(x)
    nz = x > 0
    K[nz] = 2.0 * special.j1(x[nz]) / x[nz]
    return K


def smooth_source(I, pixel_km: float, radius_km: float):
    """I_ext = P_r * h: periodic convolution with the projected stellar disk (Eq. iprh)."""
    K = source_kernel(I.shape[0], pixel_km, radius_km)
    return np.real(ifft2(fft2(I) * K))


# ---------------------------------------------------------------------------
# Light curves and modulation index (Sect. 3.3, Sect. 4)
# ---------------------------------------------------------------------------
def track_positions(track, n_samples: int):
    """Sample positions (pixel units) along a straight track (Sect. 3.3).

    track = (x0, y0, theta, ds); sample s at (x0 + s ds cos theta, y0 + s ds sin theta).
    Pixel (ix, iy) sits at integer coordinates (ix, iy).
    """
    x0, y0, th, ds = (float(v) for v in track)
    s = np.arange(n_samples, dtype=np.float64)
    return x0 + s * ds * math.cos(th), y0 + s * ds * math.sin(th)


def bilinear_periodic(I, x, y):
    """Bilinear interpolation of I[iy, ix] at (x, y) with periodic wrap (Reading R10)."""
    n_y, n_x = I.shape
    fx0 = np.floor(x)
    fy0 = np.floor(y)
    tx = x - fx0
    ty = y - fy0
    ix0 = np.mod(fx0.astype(np.int64), n_x)
    iy0 = np.mod(fy0.astype(np.int64), n_y)
    ix1 = np.mod(ix0 + 1, n_x)
    iy1 = np.mod(iy0 + 1, n_y)
    return ((1 - tx) * (1 - ty) * I[iy0, ix0] + tx * (1 - ty) * I[iy0, ix1]
            + (1 - tx) * ty * I[iy1, ix0] + tx * ty * I[iy1, ix1])


def lightcurves(I, tracks, n_samples: int):
    """Light curves: the pattern sampled along straight tracks at constant speed (Sect. 3.3)."""
    out = np.empty((len(tracks), n_samples))
    for t, tr in enumerate(tracks):
        x, y = track_positions(tr, n_samples)
        out[t] = bilinear_periodic(I, x, y)
    return out


def modulation_index(x):
    """m = sigma_I / mean(I) with the population standard deviation (Sect. 4, Reading R11)."""
    x = np.asarray(x, dtype=np.float64)
    return float(np.std(x) / x.mean())


def diffraction_radius_km(p: ScreenParams, lambda_nm: float) -> float:
    """R_diff(lambda) for a fixed screen: phi scales as lambda_ref/lambda, so D = (r/R_diff)^(beta-2)
    gives R_diff(lambda) = R_diff(lambda_ref) (lambda/lambda_ref)^(2/(beta-2)) (6/5 for Kolmogorov, Sect. 3.2.4)."""
    return p.r_diff_km * (lambda_nm / p.lambda_ref_nm) ** (2.0 / (p.beta - 2.0))


def refraction_radius_km(p: ScreenParams, lambda_nm: float) -> float:
    """R_ref = lambda z_0 / R_diff(lambda) (Eq. Rrefraction)."""
    return lambda_nm * KM_PER_NM * p.z_pc * KM_PER_PC / diffraction_radius_km(p, lambda_nm)


def fiducial_margin_km(p: ScreenParams) -> float:
    """Margin of the fiducial zone: L_m + R_ref/2 + R_s (Sect. 3.2.1, 3.2.3), at lambda = p.lambda_nm."""
    return (taper_margin_km(p, p.lambda_nm) + 0.5 * refraction_radius_km(p, p.lambda_nm)
            + p.source_radius_km)


def fiducial_slice(p: ScreenParams):
    """Index range [i0, i1) of pixels whose centres lie at least the fiducial margin from both borders.

    Whole map when the taper is off or the zone would be empty (Reading R11).
    Returns (i0, i1, flagged_whole_map).
    """
    n = p.n
    if p.margin_km == 0.0:
        return 0, n, False
    m = fiducial_margin_km(p)
    x = (np.arange(n) + 0.5) * p.pixel_km
    inside = np.nonzero((x >= m) & (x <= n * p.pixel_km - m))[0]
    if inside.size == 0:
        return 0, n, True
    return int(inside[0]), int(inside[-1]) + 1, False


def modulation_index_map(I, p: ScreenParams):
    """Modulation index of an intensity map over its fiducial zone (Sect. 4.1, Reading R11)."""
    i0, i1, _ = fiducial_slice(p)
    return modulation_index(I[i0:i1, i0:i1])


# ---------------------------------------------------------------------------
# Modulation-index sweeps (Sect. 4.1): Eq. xparam and the number of refractive
# regions in the fiducial zone
# ---------------------------------------------------------------------------
R_SUN_KM = 695700.0


def xparam_m(r_diff_km: float, lambda_nm: float, z0_pc: float, source_radius_km: float) -> float:
    """Eq. xparam, first form: m ~ (R_diff / R_F)^(1/3) (R_ref / (2 pi R_s))^(7/6), with
    R_F = sqrt(lambda z_0 / 2 pi) and R_ref = lambda z_0 / R_diff (strong, quenched regime)."""
    lz = lambda_nm * KM_PER_NM * z0_pc * KM_PER_PC
    r_f = math.sqrt(lz / (2.0 * math.pi))
    r_ref = lz / r_diff_km
    return (r_diff_km / r_f) ** (1.0 / 3.0) * (r_ref / (2.0 * math.pi * source_radius_km)) ** (7.0 / 6.0)


def xparam_m_numeric(r_diff_km: float, lambda_nm: float, z0_pc: float, r_s_over_z1_rsun_per_10kpc: float,
                     coefficient: float = 0.035) -> float:
    """Eq. xparam, numerical form: 0.035 (lambda/1 um) (z_0/1 kpc)^(-1/6) (R_diff/1000 km)^(-5/6)
    ((r_s/z_1) / (R_sun/10 kpc))^(-7/6)."""
    return (coefficient * (lambda_nm / 1000.0) * (z0_pc / 1000.0) ** (-1.0 / 6.0)
            * (r_diff_km / 1000.0) ** (-5.0 / 6.0) * r_s_over_z1_rsun_per_10kpc ** (-7.0 / 6.0))


def refractive_regions(p: ScreenParams) -> float:
    """N_R ~ d^2 / R_ref^2 (Sect. 4.1): R_ref-size regions in the fiducial zone of side d
    (0 when the zone is empty)."""
    i0, i1, whole = fiducial_slice(p)
    if whole and p.margin_km != 0.0:
        return 0.0
    d = (i1 - i0) * p.pixel_km
    return d * d / refraction_radius_km(p, p.lambda_nm) ** 2


# ---------------------------------------------------------------------------
# Light-curve time analysis (Sect. 5): power spectra and the decorrelation of
# two telescopes
# ---------------------------------------------------------------------------
def periodogram(curves):
    """One-sided periodogram of each light curve, P_k = |sum_s (c_s - mean c) e^{-2 pi i k s / n}|^2 / n
    for k = 0..n/2 (the time power spectrum whose slope breaks near 1/t_ref, Sect. 5)."""
    c = np.atleast_2d(np.asarray(curves, dtype=np.float64))
    x = c - c.mean(axis=1, keepdims=True)
    return np.abs(np.fft.rfft(x, axis=1)) ** 2 / c.shape[1]


def pearson(a, b):
    """Correlation coefficient of light curves a and b (rows): how far two telescopes' curves
    decorrelate (Sect. 5)."""
    a = np.atleast_2d(np.asarray(a, dtype=np.float64))
    b = np.atleast_2d(np.asarray(b, dtype=np.float64))
    da = a - a.mean(axis=1, keepdims=True)
    db = b - b.mean(axis=1, keepdims=True)
    return (da * db).sum(axis=1) / np.sqrt((da * da).sum(axis=1) * (db * db).sum(axis=1))


def parallel_tracks(track, separations_px):
    """Tracks parallel to `track` (x0, y0, theta, ds), offset perpendicularly by each separation
    (pixels): the sections two telescopes a distance apart sweep (Sect. 5)."""
    x0, y0, th, ds = track
    sep = np.asarray(separations_px, dtype=np.float64)
    return np.stack([x0 - sep * math.sin(th), y0 + sep * math.cos(th), np.full(sep.shape, th),
                     np.full(sep.shape, ds)], axis=1)


# ---------------------------------------------------------------------------
# Whole forward path and its adjoint (gradient of a light-curve misfit)
# ---------------------------------------------------------------------------
def forward(p: ScreenParams, lambdas_nm, tracks, n_samples: int, weights=None, phi=None):
    """Screen -> passband intensity -> source smoothing -> light curves.  Returns (phi, I, curves)."""
    if phi is None:
        phi = make_screen(p)
    I = sum_passband(phi, p, lambdas_nm, weights)
    if p.source_radius_km > 0.0:
        I = smooth_source(I, p.pixel_km, p.source_radius_km)
    return phi, I, lightcurves(I, tracks, n_samples)


def misfit_loss(curves, target):
    """L = mean squared misfit between simulated and target light curves."""
    return float(np.mean((curves - target) ** 2))


def bilinear_periodic_adjoint(shape, x, y, g):
    """Transpose of bilinear_periodic: scatter g with the bilinear weights (periodic)."""
    n_y, n_x = shape
    out = np.zeros(shape)
    fx0 = np.floor(x)
    fy0 = np.floor(y)
    tx = x - fx0
    ty = y - fy0
    ix0 = np.mod(fx0.astype(np.int64), n_x)
    iy0 = np.mod(fy0.astype(np.int64), n_y)
    ix1 = np.mod(ix0 + 1, n_x)
    iy1 = np.mod(iy0 + 1, n_y)
    np.add.at(out, (iy0, ix0), (1 - tx) * (1 - ty) * g)
    np.add.at(out, (iy0, ix1), tx * (1 - ty) * g)
    np.add.at(out, (iy1, ix0), (1 - tx) * ty * g)
    np.add.at(out, (iy1, ix1), tx * ty * g)
    return out


def misfit_gradient(p: ScreenParams, phi, lambdas_nm, tracks, n_samples: int, target, weights=None,
                    return_curves: bool = False):
    """Gradient of the light-curve misfit w.r.t. every screen pixel and R_diff (reverse mode).

    Chain, last step first:
      dL/dc   = 2 (c - t) / M
      dL/dI   = B^T dL/dc, then the disk filter K (real and even, so self-adjoint)
      G_out   = 2 w_l (dL/dI) A_out                           (complex gradient of |A|^2)
      G_in    = IDFT(DFT(G_out) conj(H))                      (adjoint of the unitary propagator)
      dL/dphi = sum_l s_l Im(conj(A_in) G_in)                 (A_in = T exp(i s phi))
      dL/dR_diff = ((2 - beta) / (2 R_diff)) sum phi dL/dphi  (phi ~ R_diff^((2-beta)/2), fixed seed)
    Returns (loss, dL/dphi, dL/dR_diff), and the forward pass's curves c after them when
    return_curves is set.
    """
    lambdas_nm = np.asarray(lambdas_nm, dtype=np.float64)
    if weights is None:
        weights = np.full(lambdas_nm.shape, 1.0 / lambdas_nm.size)
    _, I, curves = forward(p, lambdas_nm, tracks, n_samples, weights, phi=phi)
    M = curves.size
    gc = 2.0 * (curves - target) / M
    gI = np.zeros((p.n, p.n))
    for t, tr in enumerate(tracks):
        x, y = track_positions(tr, n_samples)
        gI += bilinear_periodic_adjoint((p.n, p.n), x, y, gc[t])
    if p.source_radius_km > 0.0:
        gI = smooth_source(gI, p.pixel_km, p.source_radius_km)
    gphi = np.zeros((p.n, p.n))
    for lam, w in zip(lambdas_nm, weights):
        s = p.lambda_ref_nm / lam
        a_in = screen_field(phi, p, lam)
        a_out = propagate_field(a_in, p.pixel_km, lam, p.z_pc)
        g_out = 2.0 * w * gI * a_out
        H = transfer_function(p.n, p.pixel_km, lam, p.z_pc)
        g_in = ifft2(fft2(g_out) * np.conj(H))
        gphi += s * np.imag(np.conj(a_in) * g_in)
    g_rdiff = (2.0 - p.beta) / (2.0 * p.r_diff_km) * float(np.sum(phi * gphi))
    if return_curves:
        return misfit_loss(curves, target), gphi, g_rdiff, curves
    return misfit_loss(curves, target), gphi, g_rdiff
