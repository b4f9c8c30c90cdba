"""FP64 CPU oracle for spectral correlation density (SCD) estimation: FAM and SSCA.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the CUDA
path is checked against.  Only the test suite, the smoke check of the package entry
file and the CPU-baseline leg of the benchmark may import it; the library never does,
and it imports nothing from the library.  It shares no code with the CUDA path.

Everything is complex128 / float64.  Inputs arrive as complex64 signals and float32
windows (the same bits the GPU sees) and are promoted, so a parity check measures only
the GPU's arithmetic error.  Two modes share nothing but the index conventions:

  * mode="direct": every DFT is an explicit O(M^2) sum, written as a product with the
    DFT matrix exp(-i*2*pi*((j*k) mod M)/M) built from exact integer indices;
  * mode="fft": the same sums evaluated with numpy.fft (a library primitive).

Conventions (fs = 1; all axes stored "fftshifted"):
  * channel k in [-Np/2, Np/2) is stored at kh = k + Np/2   (all Np channels, the
    down-conversion phase being Np-periodic in k);
  * FAM second-FFT bin q in [-P/2, P/2) is stored at qh = q + P/2;
  * SSCA bin q in [-N/2, N/2) is stored at sh = q + N/2;
  * P and N need not be powers of two; for an odd size M the signed bins are
    q in [-(M-1)/2, (M-1)/2], stored at q + floor(M/2) (the order numpy's fftshift gives:
    the zero bin at floor(M/2), the most negative bin first);
  * W_M^j = exp(-i*2*pi*j/M); every phase index is an exact integer product reduced
    to its non-negative residue mod M before it becomes an angle;
  * windows g, g_d of the SCD low-pass (Sec. II-A, II-B, II-C) are rectangular (= 1);
  * no 1/N or 1/P scaling anywhere: raw sums.

Besides the auto estimate (the paper's case) both estimators take a second signal y
(the cross estimate of Sec. II-A, Eq. II.A-SCD function) and a conjugate form (the
product without the conjugation); alpha profiles are the column maxima of the maps.

Pins (tests/test_oracle_*.py): the default symmetric Hamming window against scipy's
hamming(sym=True) and its closed forms (0.08 endpoints, symmetry, peak, sum), the
Dolph-Chebyshev window against scipy's chebwin, brute-force triple sums on tiny inputs (auto, cross and
conjugate; power-of-two and other sizes, odd ones included), direct vs fft mode, cross Hermitian symmetry, the conjugate estimate as a
cross estimate against conj(y) with the l axis reversed, the averaged-periodogram identity at alpha = 0 (also against scipy's Welch
estimate), the lag-windowed correlogram at alpha = 0 for SSCA, exact conjugate
symmetry (FAM), exact channel-shift invariance, |c|^2 scaling, the closed-form FAM
response to sums of channel-centred tones, cyclic-feature locations of BPSK, and the
white-noise floor.  The paper prints no worked numeric example, so agreement with the
paper's own output values is "parity unpinned" (every function here is pinned by the
identities above instead).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "hamming_window",
    "chebyshev_window",
    "chebyshev_window64",
    "input_scale",
    "twiddle",
    "fam_demodulates",
    "fam",
    "fam_pairs",
    "ssca_demodulates",
    "ssca_cdp",
    "ssca_strip",
    "ssca",
    "fam_map",
    "ssca_map",
    "fam_map_coords",
    "ssca_map_coords",
    "fam_alpha_profile",
    "ssca_alpha_profile",
]


# ----------------------------------------------------------------------------- helpers
def hamming_window(Np: int) -> np.ndarray:
    """Symmetric Hamming window a[n] = 0.54 - 0.46 cos(2 pi n / (Np - 1)), rounded to
    float32 (the window bits both sides consume when the caller passes none)."""
    n = np.arange(Np, dtype=np.float64)
    return (0.54 - 0.46 * np.cos(2.0 * np.pi * n / (Np - 1))).astype(np.float32)


def chebyshev_window64(Np: int, atten_db: float) -> np.ndarray:
    """Dolph-Chebyshev window (Algorithms 1 and 2 window the channeliser input with
    `chebwin[Np]`) in FP64: equiripple sidelobes atten_db below the main lobe.  From the
    textbook definition: the window's Np-point spectrum samples are the Chebyshev polynomial
    T_{Np-1}(x0 cos(pi k / Np)) with x0 = cosh(acosh(10^{atten/20}) / (Np - 1)); the window,
    symmetric about (Np - 1)/2, is their inverse DFT (a real cosine sum), scaled to a peak of 1.
    """
    M = Np - 1
    x0 = np.cosh(np.arccosh(10.0 ** (atten_db / 20.0)) / M)

    def cheb(x):
        x = np.asarray(x, dtype=np.float64)
        inside = np.abs(x) <= 1.0
        out = np.empty_like(x)
        out[inside] = np.cos(M * np.arccos(x[inside]))
        big = np.cosh(M * np.arccosh(np.abs(x[~inside])))
        out[~inside] = np.where((x[~inside] < 0) & (M % 2 == 1), -big, big)
        return out

    k = np.arange(1, (Np - 1) // 2 + 1, dtype=np.float64)
    Wk = cheb(x0 * np.cos(np.pi * k / Np))
    n = np.arange(Np, dtype=np.float64)
    w = cheb(np.array([x0]))[0] + 2.0 * (np.cos(2.0 * np.pi * np.outer(n - (Np - 1) / 2.0, k) / Np) @ Wk)
    return w / np.max(w)


def chebyshev_window(Np: int, atten_db: float = 100.0) -> np.ndarray:
    """chebyshev_window64 rounded to float32 (the window bits both sides consume)."""
    return chebyshev_window64(Np, atten_db).astype(np.float32)


def twiddle(M: int, idx) -> np.ndarray:
    """W_M^idx = exp(-i 2 pi idx / M) for integer idx (any sign, any size): the index is
    reduced exactly to [0, M) as an integer before it is turned into an angle."""
    j = np.mod(np.asarray(idx, dtype=np.int64), M)
    return np.exp(-2j * np.pi * (j.astype(np.float64) / M))


def _partner(x, y):
    """The second signal of a cross estimate (Sec. II-A, Eq. II.A-SCD function pairs the
    demodulates of x and y); y = None is the auto estimate, y = x."""
    if y is None:
        return x
    if np.asarray(y).shape != np.asarray(x).shape:
        raise ValueError("x and y must have the same length")
    return y


def _promote(x, a, scale: float = 1.0):
    x = np.asarray(x)
    a = np.asarray(a)
    if x.dtype != np.complex64:
        raise TypeError("x must be complex64 (the bits the GPU path consumes)")
    if a.dtype != np.float32:
        raise TypeError("window must be float32 (the bits the GPU path consumes)")
    return x.astype(np.complex128) * scale, a.astype(np.float64)


def input_scale(x, used: int, mode: int) -> float:
    """The factor the `Normalize` step of Algorithm 1 (`Framing`: the norm kernel normalises
    the input before decimation, Sec. III-A) multiplies the input by, computed in FP64 over
    the `used` samples the estimate consumes: mode 1 makes their mean power 1
    (1/sqrt(mean |x|^2)), mode 2 their peak magnitude 1 (1/max |x|), mode 0 leaves the input
    as it is.  An all-zero input is left as it is."""
    if mode == 0:
        return 1.0
    v = np.asarray(x)[:used].astype(np.complex128)
    p = np.mean(np.abs(v) ** 2) if mode == 1 else np.max(np.abs(v)) ** 2
    return 1.0 / np.sqrt(p) if p > 0 else 1.0


def _signed_channels(Np: int) -> np.ndarray:
    return np.arange(-Np // 2, Np // 2, dtype=np.int64)


def _dft_rows(blocks: np.ndarray, M: int, out_bins: np.ndarray, mode: str) -> np.ndarray:
    """sum_{j<M} blocks[..., j] W_M^{(j * b) mod M} for each requested bin b."""
    if mode == "direct":
        F = twiddle(M, np.outer(np.arange(M, dtype=np.int64), out_bins))
        return blocks @ F
    if mode == "fft":
        return np.fft.fft(blocks, axis=-1)[..., np.mod(out_bins, M)]
    raise ValueError(f"unknown mode {mode!r}")


# ----------------------------------------------------------------------------- FAM
def fam_demodulates(x, a, Np: int, L: int, P: int, mode: str = "fft", scale: float = 1.0) -> np.ndarray:
    """FAM channeliser (Sec. II-B-1, Eq. II.B-complex_demodulate_final, with the block
    framing of Algorithm 1 `Framing`: block p covers x[pL .. pL+Np-1]).

        X(p, k) = W_Np^{(k p L) mod Np} * sum_{n<Np} a[n] x[pL + n] W_Np^{(k n) mod Np}

    The first factor is the down-conversion.  `scale` multiplies the input first (input
    normalisation).  Returns complex128 [Np (kh)][P (p)].
    """
    x, a = _promote(x, a, scale)
    if x.shape[0] < (P - 1) * L + Np:
        raise ValueError("FAM needs N >= (P-1)*L + Np samples")
    n = np.arange(Np, dtype=np.int64)
    p = np.arange(P, dtype=np.int64)
    k = _signed_channels(Np)
    blocks = x[p[:, None] * L + n[None, :]] * a[None, :]          # [P][Np]
    spectra = _dft_rows(blocks, Np, k, mode)                      # [P][Np (kh)]
    down = twiddle(Np, np.outer(p * L, k))                        # W_Np^{k p L}
    return (spectra * down).T.copy()                              # [kh][p]


def _signed_bins(M: int) -> np.ndarray:
    """Signed bins of a size-M DFT in stored order: q in [-floor(M/2), M - floor(M/2)),
    q stored at q + floor(M/2) (for even M, [-M/2, M/2))."""
    return np.arange(-(M // 2), M - M // 2, dtype=np.int64)


def _fam_second_fft(z: np.ndarray, P: int, mode: str) -> np.ndarray:
    """S(q) = sum_{p<P} z(p) W_P^{(q p) mod P} for the signed bins q of _signed_bins(P),
    stored at q + floor(P/2)."""
    return _dft_rows(z, P, _signed_bins(P), mode)


def fam_pairs(x, a, Np: int, L: int, P: int, kh, lh, mode: str = "fft", y=None,
              conjugate: bool = False) -> np.ndarray:
    """FAM estimate for selected channel pairs (kh[i], lh[i]) (Sec. II-B-2,
    Eq. II.B-SCD_function_FAM with g_d = 1):

        S(k, l, q) = sum_{p<P} X(p, k) conj(Y(p, l)) W_P^{(q p) mod P}

    i.e. the conjugate multiplication followed by the P-point FFT.  Y is the channeliser
    output of y (Eq. II.A-SCD function's cross form; y = None: Y = X, the auto estimate).
    conjugate=True forms the conjugate estimate: the product X(p, k) Y(p, l) without the
    conjugation, which correlates x near f_k with y near f_l in the conjugate sense
    (alpha = f_k + f_l + q/(P L), f = (f_k - f_l)/2).  Returns complex128 [len(kh)][P (qh)].
    """
    X = fam_demodulates(x, a, Np, L, P, mode)
    Y = X if y is None else fam_demodulates(_partner(x, y), a, Np, L, P, mode)
    kh = np.asarray(kh, dtype=np.int64)
    lh = np.asarray(lh, dtype=np.int64)
    second = Y[lh, :] if conjugate else np.conj(Y[lh, :])
    z = X[kh, :] * second                                          # [pairs][P]
    return _fam_second_fft(z, P, mode)


def fam(x, a, Np: int, L: int, P: int, mode: str = "fft", y=None, conjugate: bool = False,
        normalise: int = 0) -> np.ndarray:
    """Full FAM estimate, complex128 [Np (kh)][Np (lh)][P (qh)] (y, conjugate: as in
    fam_pairs; normalise: the input normalisation of input_scale, auto estimate only)."""
    if normalise and y is not None:
        raise ValueError("input normalisation is defined for the auto estimate")
    X = fam_demodulates(x, a, Np, L, P, mode, input_scale(x, (P - 1) * L + Np, normalise))
    Y = X if y is None else fam_demodulates(_partner(x, y), a, Np, L, P, mode)
    second = Y if conjugate else np.conj(Y)
    out = np.empty((Np, Np, P), dtype=np.complex128)
    for kh in range(Np):                                          # one channel row at a time
        z = X[kh][None, :] * second                               # [lh][p]
        out[kh] = _fam_second_fft(z, P, mode)
    return out


# ----------------------------------------------------------------------------- SSCA
def ssca_demodulates(x, a, Np: int, n, channels=None, mode: str = "fft", scale: float = 1.0) -> np.ndarray:
    """SSCA channeliser at hop 1 (Sec. II-C; the complex demodulate of Sec. II-A,
    Eq. II.A-complex demodulate, centred on sample n, with the window spanning
    x[n - Np/2 .. n + Np/2 - 1] and x taken as zero outside [0, N)):

        X_T(n, k) = W_Np^{(k s) mod Np} * sum_{r<Np} a[r] x[s + r] W_Np^{(k r) mod Np},
        s = n - Np/2.

    `scale` multiplies the input first (input normalisation).  Returns complex128
    [len(n)][len(channels)] (channels are stored indices kh).
    """
    x, a = _promote(x, a, scale)
    N = x.shape[0]
    n = np.asarray(n, dtype=np.int64)
    kh = np.arange(Np, dtype=np.int64) if channels is None else np.asarray(channels, np.int64)
    k = kh - Np // 2
    s = n - Np // 2
    m = s[:, None] + np.arange(Np, dtype=np.int64)[None, :]       # absolute sample index
    inside = (m >= 0) & (m < N)
    blocks = np.where(inside, x[np.clip(m, 0, N - 1)], 0.0) * a[None, :]
    spectra = _dft_rows(blocks, Np, k, mode)                      # [n][ch]
    down = twiddle(Np, np.outer(s, k))                            # W_Np^{k s}
    return spectra * down


def ssca_cdp(x, a, Np: int, n, channels=None, mode: str = "fft", y=None,
             conjugate: bool = False, scale: float = 1.0) -> np.ndarray:
    """Channel-data product of Sec. II-C, Eq. Xg with g = 1:
    X_g(n, k) = X_T(n, k) conj(y[n]), y = x for the auto estimate (Sec. II-C multiplies
    the demodulate by the conjugated second signal).  conjugate=True multiplies by y[n]
    itself (the conjugate estimate).  Returns complex128 [len(channels)][len(n)]."""
    n = np.asarray(n, dtype=np.int64)
    XT = ssca_demodulates(x, a, Np, n, channels, mode, scale)     # [n][ch]
    yn = np.asarray(_partner(x, y)).astype(np.complex128)[n] * scale
    second = yn if conjugate else np.conj(yn)
    return (XT * second[:, None]).T


def ssca_strip(Xg_row: np.ndarray, mode: str = "fft") -> np.ndarray:
    """N-point strip transform of one channel (Eq. II.B-SSCA_auto, time origin at the first
    sample): S(q) = sum_{n<N} X_g(n) W_N^{(q n) mod N}, q in [-N/2, N/2) stored at q + N/2
    (any N: the signed bins of _signed_bins(N))."""
    N = Xg_row.shape[-1]
    q = _signed_bins(N)
    if mode == "direct":
        if N > 4096:
            raise ValueError("direct SSCA strip DFT is limited to N <= 4096")
        return Xg_row @ twiddle(N, np.outer(np.arange(N, dtype=np.int64), q))
    return np.fft.fft(Xg_row, axis=-1)[..., np.mod(q, N)]


def ssca(x, a, Np: int, mode: str = "fft", channels=None, chunk: int = 1 << 13, y=None,
         conjugate: bool = False, normalise: int = 0) -> np.ndarray:
    """SSCA estimate (Sec. II-C, Eq. Xg and Eq. II.B-SSCA_auto, with g = 1 and the
    time origin at the first sample):

        X_g(n, k) = X_T(n, k) conj(y[n])          (y = x: the auto estimate)
        S(k, q)   = sum_{n<N} X_g(n, k) W_N^{(q n) mod N},   q in [-N/2, N/2)

    alpha = k/Np + q/N and f = (k/Np - q/N)/2.  conjugate=True uses y[n] unconjugated;
    the bin then correlates x at f_k with y at q/N in the conjugate sense, whose
    alpha = f_k + q/N and f = (f_k - q/N)/2 are the same coordinates.  Returns complex128
    [len(channels)][N (sh)], sh = q + N/2.
    """
    N = np.asarray(x).shape[0]
    if normalise and y is not None:
        raise ValueError("input normalisation is defined for the auto estimate")
    scale = input_scale(x, N, normalise)                          # input normalisation (Algorithm 1)
    kh = np.arange(Np, dtype=np.int64) if channels is None else np.asarray(channels, np.int64)
    Xg = np.empty((kh.shape[0], N), dtype=np.complex128)          # channel-major CDP
    for n0 in range(0, N, chunk):                                 # channeliser in chunks of time
        n = np.arange(n0, min(N, n0 + chunk), dtype=np.int64)
        Xg[:, n0:n0 + n.shape[0]] = ssca_cdp(x, a, Np, n, kh, mode, y, conjugate, scale)
    if mode == "direct":
        return ssca_strip(Xg, mode)                               # one DFT-matrix product
    out = np.empty_like(Xg)
    for i in range(kh.shape[0]):                                  # one channel row at a time
        out[i] = ssca_strip(Xg[i], mode)
    return out


# ----------------------------------------------------------------------------- maps
def fam_map_coords(Np: int, L: int, P: int, conjugate: bool = False):
    """Kept FAM cells and their (f, alpha) grid positions.

    Algorithm 1 (`FFT2`) keeps only the central half of each P-point output.  Here the
    kept band is q in [-Q, Q) with Q = P*L/Np, which equals [-P/4, P/4) when L = Np/4.
    f = (f_k + f_l)/2 and alpha = f_k - f_l + q/(P L) (Sec. II-B-2), so with integer
    grid indices fh = k + l + Np (f = (fh - Np)/(2 Np)) and
    ah = (k - l) Q + q + P L (alpha = (ah - P L)/(P L)).
    The conjugate estimate has f = (f_k - f_l)/2 and alpha = f_k + f_l + q/(P L):
    fh = k - l + Np, ah = (k + l) Q + q + P L; the cells with alpha < -1 (ah < 0, only
    at k = l = -Np/2) fall outside the principal domain and are not kept.
    Returns int64 arrays kh, lh, qh, fh, ah (one entry per kept cell).
    """
    if (P * L) % Np or 2 * L > Np:
        raise ValueError("FAM map needs P*L divisible by Np and L <= Np/2")
    Q = P * L // Np
    k = _signed_channels(Np)
    kk, ll, qq = np.meshgrid(k, k, np.arange(-Q, Q, dtype=np.int64), indexing="ij")
    kk, ll, qq = kk.ravel(), ll.ravel(), qq.ravel()
    if not conjugate:
        return (kk + Np // 2, ll + Np // 2, qq + P // 2, kk + ll + Np, (kk - ll) * Q + qq + P * L)
    ah = (kk + ll) * Q + qq + P * L
    keep = ah >= 0
    return (kk[keep] + Np // 2, ll[keep] + Np // 2, qq[keep] + P // 2, (kk - ll + Np)[keep], ah[keep])


def fam_map(S: np.ndarray, Np: int, L: int, P: int, power: int = 1, conjugate: bool = False) -> np.ndarray:
    """Scatter |S|^power of the kept FAM cells onto the float64 [2 Np][2 P L] grid;
    cells that no (k, l, q) reaches stay 0."""
    kh, lh, qh, fh, ah = fam_map_coords(Np, L, P, conjugate)
    grid = np.zeros((2 * Np, 2 * P * L), dtype=np.float64)
    grid[fh, ah] = np.abs(S[kh, lh, qh]) ** power
    return grid


def ssca_map_coords(N: int, Np: int):
    """SSCA (f, alpha) positions of every output cell (Sec. II-C: alpha = f_k + q/N,
    f = (f_k - q/N)/2; the same mapping as Sec. III-B-1's SSCA_2DFFT formula with
    the stored index M1 m2' + m1' = q + N/2).

    ah = k N/Np + q + N             (alpha = (ah - N)/N, in [-1, 1))
    fh = floor((k N/Np - q + N) / (2 N/Np))   (f in [fh, fh+1) * 1/Np - 1/2)
    The channel centres k/Np fall on the alpha grid 1/N only when Np divides N, so the map
    needs that.  Returns int64 arrays kh, sh, fh, ah for all Np*N cells.
    """
    if N % Np:
        raise ValueError("SSCA map needs Np to divide N")
    k = _signed_channels(Np)
    q = np.arange(-N // 2, N // 2, dtype=np.int64)
    kk, qq = np.meshgrid(k, q, indexing="ij")
    kk, qq = kk.ravel(), qq.ravel()
    D = N // Np
    ah = kk * D + qq + N
    fh = np.floor_divide(kk * D - qq + N, 2 * D)
    return kk + Np // 2, qq + N // 2, fh, ah


def ssca_map(S: np.ndarray, N: int, Np: int, power: int = 1) -> np.ndarray:
    """Scatter |S|^power onto the float64 [Np][2N] grid; unreached cells stay 0."""
    kh, sh, fh, ah = ssca_map_coords(N, Np)
    grid = np.zeros((Np, 2 * N), dtype=np.float64)
    grid[fh, ah] = np.abs(S[kh, sh]) ** power
    return grid


# ----------------------------------------------------------------------------- alpha profiles
def fam_alpha_profile(S: np.ndarray, Np: int, L: int, P: int, power: int = 1,
                      conjugate: bool = False) -> np.ndarray:
    """Cycle-frequency profile: for every alpha column ah of the FAM map, the largest
    |S|^power over f (the feature vector the paper's RFML motivation, Sec. I, extracts
    from the SCD).  Columns that no cell reaches are 0.  Returns float64 [2 P L]."""
    return fam_map(S, Np, L, P, power, conjugate).max(axis=0)


def ssca_alpha_profile(S: np.ndarray, N: int, Np: int, power: int = 1) -> np.ndarray:
    """Cycle-frequency profile of the SSCA map: largest |S|^power over f per alpha column
    ah.  Returns float64 [2 N]."""
    return ssca_map(S, N, Np, power).max(axis=0)
