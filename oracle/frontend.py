"""SFT front end: from short Fourier transforms to the heterodyned series
(FP64, test oracle; Sec. III.B).

TEST INFRASTRUCTURE: only tests/, the smoke check and the bench's CPU
baseline may use this module; the library never does.

The steps of the summary in Sec. III.B.7, after the SFTs exist (step 1, the
data product of Eq. e25, X_{alpha,k} = sum_j x_{alpha,j} e^{-2 pi i j k / N}):

2. normalise every SFT by its noise (Eq. dimlessSFTs1): X^ = X / sqrt(S)
   with S a running median of |X|^2 over w bins divided by ln 2 (the
   median of an exponential variable is ln 2 times its mean), so that
   E|X^|^2 = 1 per bin; the window is truncated at the ends of the stored
   band and an even count takes its lower median;
3. split the SFTs into contiguous runs (chunks): SFT alpha + 1 starts one
   SFT length after SFT alpha, to within 1e-6 of that length (a bin whose
   noise estimate of step 2 is zero is set to zero);
4. merge each chunk of M SFTs into the long time-baseline transform with
   the truncated Dirichlet kernel, Eq. e9:
     X_b = sum_alpha e^{-2 pi i b alpha / M}
           sum_{k = k* - dk}^{k* + dk} X_{alpha,k} P_{b,k},   k* = floor(b / M),
     P_{b,k} = sin y / y - i (1 - cos y) / y,   y = 2 pi (b / M - k)
   (Eq. e75's large-N form; P = 1 at y = 0; the printed P_{alpha,k} of
   Eq. e9 is read as P_{b,k}, the kernel defined just above it);
5. keep the band of N_out = N1 M long-transform bins around b_h = k_h M
   (Sec. III.B.4: the heterodyne bin relabelled as DC), weight it with a
   Tukey window (Sec. III.B.5) and inverse transform it:
     z[n] = 1 / sqrt(M N_out) sum_{m=-N_out/2}^{N_out/2-1} w_m X_{b_h+m} e^{2 pi i m n / N_out},
   samples n dt_out after the chunk start, dt_out = T_SFT / N1; the scale
   makes the noise variance of z the mean square of the window when the
   normalisation of step 2 is exact;
6. multiply by the chunk's phase factor (Eq. hetStartCorr with the sign of
   the heterodyne x_h = x e^{-2 pi i f_h (t - t_s)}, i.e.
   e^{-2 pi i f_h (t_c - t_s)}), optionally taper its ends in time, and
   place it at its offset (t_c - t_s) / dt_out of the output; samples of no
   chunk (gaps) are zero (Sec. III.B.6).

Everything here is plain loops and numpy.fft, slow and literal.
"""
from __future__ import annotations

import math

import numpy as np


def running_median_psd(X, w):
    """S_{alpha,k}: running median of |X|^2 over the w bins centred on k
    (truncated at the band ends; lower median for an even count) / ln 2."""
    P = np.abs(np.asarray(X, np.complex128)) ** 2
    n_sft, K = P.shape
    h = w // 2
    S = np.empty_like(P)
    for k in range(K):
        lo, hi = max(0, k - h), min(K, k + h + 1)
        win = np.sort(P[:, lo:hi], axis=1)
        S[:, k] = win[:, (hi - lo - 1) // 2]
    return S / math.log(2.0)


def normalize(X, w):
    """Eq. dimlessSFTs1 (w = 0: no normalisation).  A bin whose noise
    estimate is zero (its window holds zeros only, e.g. an SFT of zeros)
    carries no information and is set to zero."""
    X = np.asarray(X, np.complex128)
    if w == 0:
        return X.copy()
    S = running_median_psd(X, w)
    out = np.zeros_like(X)
    ok = S > 0
    out[ok] = X[ok] / np.sqrt(S[ok])
    return out


def chunks(t_sft, t_len, rtol=1e-6):
    """Contiguous runs of SFTs: list of (first index, count); SFT i + 1
    continues the run when it starts T_SFT after SFT i to within
    rtol T_SFT."""
    out = []
    a = 0
    for i in range(1, len(t_sft) + 1):
        if i == len(t_sft) or abs(t_sft[i] - t_sft[i - 1] - t_len) > rtol * t_len:
            out.append((a, i - a))
            a = i
    return out


def dirichlet(b, k, M):
    """P_{b,k} of Eq. e9 (large-N form of Eq. e75)."""
    y = 2.0 * math.pi * (b / M - k)
    if y == 0.0:
        return 1.0 + 0.0j
    return complex(math.sin(y) / y, -(1.0 - math.cos(y)) / y)


def merge(Xh, k_lo, b_values, dk):
    """Eq. e9 for one chunk: Xh (M, K) normalised SFT bins k_lo .. k_lo+K-1;
    returns X_b for each b in b_values (absolute long-transform bins)."""
    M, K = Xh.shape
    out = np.zeros(len(b_values), np.complex128)
    for i, b in enumerate(b_values):
        ks = b // M
        acc = 0.0j
        for alpha in range(M):
            ph = np.exp(-2j * math.pi * ((b * alpha) % M) / M)
            s = 0.0j
            for k in range(ks - dk, ks + dk + 1):
                s += Xh[alpha, k - k_lo] * dirichlet(b, k, M)
            acc += ph * s
        out[i] = acc
    return out


def tukey(n, frac):
    """Tukey window of n points over x = (i + 1/2) / n: a raised-cosine rise
    over the first frac / 2 of the band, flat, and the mirrored fall."""
    x = (np.arange(n) + 0.5) / n
    w = np.ones(n)
    if frac <= 0:
        return w
    e = frac / 2.0
    lo = x < e
    hi = x > 1.0 - e
    w[lo] = 0.5 * (1.0 - np.cos(math.pi * x[lo] / e))
    w[hi] = 0.5 * (1.0 - np.cos(math.pi * (1.0 - x[hi]) / e))
    return w


def chunk_series(Xh, k_lo, k_h, n1, dk, tukey_frac, b_merge=None):
    """Steps 4-5 for one chunk: z[n], n = 0 .. N1 M - 1."""
    M = Xh.shape[0]
    n_out = n1 * M
    m = np.arange(-n_out // 2, n_out // 2)
    b = k_h * M + m
    Xb = merge(Xh, k_lo, b, dk) if b_merge is None else b_merge(Xh, k_lo, b, dk)
    spec = Xb * tukey(n_out, tukey_frac)
    # z[n] = sum_m spec_m e^{2 pi i m n / N_out}: index m taken mod N_out
    z = np.fft.ifft(np.fft.ifftshift(spec)) * n_out
    return z / math.sqrt(M * n_out)


def sft_to_series(X, t_sft, d, t_start, n_out, merge_fn=None):
    """Steps 2-6: X (n_sft, K) stored SFT bins k_lo .. k_lo+K-1 of SFTs
    starting at t_sft; d: an object with sft_len, dt_raw, k_lo, k_het,
    band_bins, dirichlet_terms, median_window, tukey_frac, edge_taper.
    Returns the complex series of n_out samples at dt_out from t_start."""
    t_len = d.sft_len * d.dt_raw
    dt_out = t_len / d.band_bins
    f_h = d.k_het / t_len
    Xh = normalize(X, d.median_window)
    x = np.zeros(n_out, np.complex128)
    for a, M in chunks(t_sft, t_len):
        z = chunk_series(Xh[a:a + M], d.k_lo, d.k_het, d.band_bins, d.dirichlet_terms, d.tukey_frac,
                         b_merge=merge_fn)
        tc = t_sft[a]
        cyc = f_h * (tc - t_start)
        z = z * np.exp(-2j * math.pi * (cyc - math.floor(cyc)))
        if d.edge_taper > 0:
            e = min(d.edge_taper, len(z) // 2)
            r = 0.5 * (1.0 - np.cos(math.pi * (np.arange(e) + 0.5) / e))
            z[:e] *= r
            z[len(z) - e:] *= r[::-1]
        off = int(round((tc - t_start) / dt_out))
        x[off:off + len(z)] = z
    return x
