"""Number-format definitions used by the precision variants — TEST INFRASTRUCTURE ONLY.

Everything here is written from the published definitions of the formats,
not from any GPU code:

* bfloat16: IEEE-754 binary32 with the low 16 fraction bits dropped (8
  significant bits, same exponent range); conversion rounds to nearest, ties
  to even.
* FP8 E4M3 (the OCP 8-bit floating point "E4M3" encoding): 1 sign bit, 4
  exponent bits with bias 7, 3 fraction bits; exponent field 0 encodes
  subnormals ``m/8 * 2^-6``; there are no infinities and only
  ``S.1111.111`` is NaN, so the largest finite magnitude is 448.  Conversion
  here is round-to-nearest-even with saturation to +-448 ("satfinite").
* Per-tensor fp8 scaling (the BF16/FP8 precision study): ``s = 448 / amax``
  (``s = 1`` when amax is 0), ``q = e4m3(x * s)``, and the dequantisation
  factor applied to the FP32 accumulator is ``1 / s``.
* Two-piece bf16 split (3xBF16): ``hi = bf16(x)``, ``lo = bf16(x - hi)``; the
  product is ``hi_a*hi_b + hi_a*lo_b + lo_a*hi_b`` (the ``lo*lo`` term is
  dropped).
* TF32 (the tensor cores' 19-bit float: 8 exponent, 10 fraction bits):
  rounding to nearest with ties away from zero; the two-piece TF32 split
  ``hi = tf32(x)``, ``lo = tf32(x - hi)`` and its three products.
* Relative Frobenius error ``||C - C_ref||_F / ||C_ref||_F``.

All rounding that decides a bit pattern is done in float32 where the GPU
does it in float32 (the scale, the product ``x*s``, the residual ``x - hi``),
so integer results (codes) can be compared bit for bit.
"""
import numpy as np

E4M3_MAX = 448.0


# ---------------------------------------------------------------- bfloat16
def bf16_bits(x):
    """Round float32 values to bfloat16 (nearest, ties to even); uint16 bits.

    Written out on the binary32 bit pattern: the kept part is the top 16 bits;
    the dropped part D (low 16 bits) is compared with the half-way point 0x8000.
    D > 0x8000 rounds up, D < 0x8000 rounds down, D == 0x8000 rounds to the
    even kept pattern.  Inputs must be finite.
    """
    x = np.ascontiguousarray(x, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("bf16_bits: finite inputs only")
    u = x.view(np.uint32).astype(np.uint64)
    kept = u >> 16
    dropped = u & 0xFFFF
    up = (dropped > 0x8000) | ((dropped == 0x8000) & ((kept & 1) == 1))
    kept = kept + up.astype(np.uint64)
    return kept.astype(np.uint16)


def bf16_to_f32(bits):
    """Exact float32 value of bfloat16 bit patterns."""
    bits = np.ascontiguousarray(bits, dtype=np.uint16)
    return (bits.astype(np.uint32) << 16).view(np.float32)


def bf16_round(x):
    """float32 -> nearest bfloat16 value, returned as float32."""
    return bf16_to_f32(bf16_bits(x))


# ---------------------------------------------------------------- FP8 E4M3
def _e4m3_table():
    """Values of the 128 non-negative codes (code 0x7F is NaN)."""
    vals = np.empty(128, dtype=np.float64)
    for code in range(128):
        e = (code >> 3) & 0xF
        f = code & 0x7
        if e == 0xF and f == 0x7:
            vals[code] = np.nan
        elif e == 0:
            vals[code] = (f / 8.0) * 2.0 ** (-6)
        else:
            vals[code] = (1.0 + f / 8.0) * 2.0 ** (e - 7)
    return vals


_E4M3_POS = _e4m3_table()


def e4m3_to_f64(codes):
    """Exact value of E4M3 byte codes (NaN for the NaN codes)."""
    codes = np.asarray(codes, dtype=np.uint8)
    mag = _E4M3_POS[codes & 0x7F]
    return np.where(codes & 0x80, -mag, mag)


def e4m3_codes(x):
    """float32 -> E4M3 codes, round to nearest even, saturating to +-448.

    For each |x| the two neighbouring representable magnitudes are found in
    the table of finite codes (0..0x7E, increasing); the nearer one wins and a
    tie goes to the code whose lowest fraction bit is 0.
    """
    x = np.asarray(x, dtype=np.float32).astype(np.float64)
    if not np.all(np.isfinite(x)):
        raise ValueError("e4m3_codes: finite inputs only")
    mag = np.minimum(np.abs(x), E4M3_MAX)
    finite = _E4M3_POS[:0x7F]                       # codes 0 .. 0x7E
    hi = np.searchsorted(finite, mag, side="left")  # finite[hi] >= mag
    hi = np.minimum(hi, 0x7E)
    lo = np.maximum(hi - 1, 0)
    d_lo = mag - finite[lo]
    d_hi = finite[hi] - mag
    pick_hi = (d_hi < d_lo) | ((d_hi == d_lo) & ((hi & 1) == 0))
    code = np.where(mag == finite[hi], hi, np.where(pick_hi, hi, lo))
    code = code.astype(np.uint8)
    # The sign bit is carried over unchanged (a negative value that rounds to
    # zero gives the negative-zero code 0x80), as in IEEE conversions.
    neg = np.signbit(x)
    return np.where(neg, code | 0x80, code).astype(np.uint8)


FP8_SCALE_MAX = np.float32(2.0 ** 126)


def fp8_scale(x):
    """Per-tensor scale ``s = min(448 / amax(|x|), 2^126)`` in float32 over the
    finite values of x (1 when amax = 0).  The cap: 448 / amax overflows float32 for amax < 448 / FLT_MAX,
    and the dequantisation factor 1 / s must stay a normal float32 (2^-126 is
    the smallest)."""
    x = np.asarray(x, dtype=np.float32)
    fin = x[np.isfinite(x)]           # non-finite values take no part in amax
    amax = np.float32(np.max(np.abs(fin))) if fin.size else np.float32(0)
    if amax == 0:
        return np.float32(1.0)
    with np.errstate(over="ignore"):
        s = np.float32(np.float32(E4M3_MAX) / amax)
    return min(s, FP8_SCALE_MAX)


def fp8_scales_pair(A, B):
    """Per-tensor scales of the two operands of one FP8 product: each
    ``min(448 / amax, 2^126)`` (``fp8_scale``); then, because the
    dequantisation 1 / (s_a s_b) is one float32 factor and must stay normal,
    when ilogb(s_a) + ilogb(s_b) exceeds 124 that excess d is taken off the
    exponents, ceil(d / 2) from s_a and floor(d / 2) from s_b (exact)."""
    sa, sb = fp8_scale(A), fp8_scale(B)
    ea = int(np.frexp(sa)[1]) - 1          # ilogb
    eb = int(np.frexp(sb)[1]) - 1
    d = ea + eb - 124
    if d > 0:
        sa = np.float32(np.ldexp(sa, -((d + 1) // 2)))
        sb = np.float32(np.ldexp(sb, -(d // 2)))
    return sa, sb


def _quantised_codes(x, s):
    """E4M3 codes of x * s (rounded to float32 first); a non-finite x gives
    the NaN code 0x7F, so infinities stay non-finite instead of saturating."""
    fin = np.isfinite(x)
    codes = e4m3_codes(np.where(fin, x * s, 0).astype(np.float32))
    return np.where(fin, codes, np.uint8(0x7F)).astype(np.uint8)


def fp8_quantize_pair(A, B):
    """Both operands of one FP8 product quantised with ``fp8_scales_pair``:
    returns (codes_a, s_a, codes_b, s_b)."""
    A = np.asarray(A, dtype=np.float32)
    B = np.asarray(B, dtype=np.float32)
    sa, sb = fp8_scales_pair(A, B)
    with np.errstate(invalid="ignore", over="ignore"):
        return _quantised_codes(A, sa), sa, _quantised_codes(B, sb), sb


def fp8_quantize(x):
    """Per-tensor quantisation: returns (codes, s) with codes = e4m3(x * s).

    The product x*s is rounded to float32 first (that is the value converted).
    The real tensor is approximated by ``e4m3_to_f64(codes) / s``.  Non-finite
    values take no part in the scale and give the NaN code 0x7F.
    """
    x = np.asarray(x, dtype=np.float32)
    s = fp8_scale(x)
    with np.errstate(invalid="ignore", over="ignore"):
        return _quantised_codes(x, s), s


# ---------------------------------------------------------------- TF32
def tf32_round(x):
    """float32 -> nearest TF32 value (10 fraction bits), ties away from zero,
    returned as float32 with the low 13 fraction bits zero.

    On the binary32 pattern: the dropped part is the low 13 bits; adding half
    of the kept unit (0x1000) to the pattern and clearing the low 13 bits
    rounds the magnitude to nearest with ties away from zero (a carry moves
    into the exponent as it should).  Finite inputs only.
    """
    x = np.ascontiguousarray(x, dtype=np.float32)
    if not np.all(np.isfinite(x)):
        raise ValueError("tf32_round: finite inputs only")
    u = x.view(np.uint32).astype(np.uint64)
    u = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return u.view(np.float32)


def split_tf32(x):
    """Two-piece TF32 split: hi = tf32(x), lo = tf32(x - hi), as float32."""
    x = np.asarray(x, dtype=np.float32)
    hi = tf32_round(x)
    lo = tf32_round((x - hi).astype(np.float32))
    return hi, lo


def split3_tf32_product(A, B, gemm):
    """hi_a*hi_b + hi_a*lo_b + lo_a*hi_b of the TF32 split, float64 via `gemm`."""
    ah, al = (p.astype(np.float64) for p in split_tf32(A))
    bh, bl = (p.astype(np.float64) for p in split_tf32(B))
    return gemm(ah, bh) + gemm(ah, bl) + gemm(al, bh)


# ---------------------------------------------------------------- 3xBF16 split
def split_bf16(x):
    """Two-piece split: (hi_bits, lo_bits) with hi = bf16(x), lo = bf16(x - hi).

    The residual x - hi is exact in float32 (hi holds the leading bits of x),
    so only the second rounding loses information.
    """
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_bits(x)
    r = (x - bf16_to_f32(hi)).astype(np.float32)
    lo = bf16_bits(r)
    return hi, lo


def split_bf16_3(x):
    """Three-piece split: hi = bf16(x), mid = bf16(x - hi), lo = bf16(x - hi - mid).

    Both residuals are formed in float32 and are exact there (each piece holds
    the leading bits of what remains), so only the roundings to bf16 lose
    information; hi + mid + lo carries ~24 significant bits of x.
    """
    x = np.asarray(x, dtype=np.float32)
    hi = bf16_bits(x)
    r1 = (x - bf16_to_f32(hi)).astype(np.float32)
    mid = bf16_bits(r1)
    r2 = (r1 - bf16_to_f32(mid)).astype(np.float32)
    lo = bf16_bits(r2)
    return hi, mid, lo


def split6_product(A, B, gemm):
    """The 6-product sum of the 3-piece split, in float64 via `gemm`:
    hi*hi + hi*mid + mid*hi + hi*lo + mid*mid + lo*hi (the mid*lo, lo*mid and
    lo*lo terms are dropped)."""
    f = lambda b: bf16_to_f32(b).astype(np.float64)
    ah, am, al = (f(p) for p in split_bf16_3(A))
    bh, bm, bl = (f(p) for p in split_bf16_3(B))
    return (gemm(ah, bh) + gemm(ah, bm) + gemm(am, bh) + gemm(ah, bl) + gemm(am, bm)
            + gemm(al, bh))


def split3_operands(A, B):
    """The three bf16 products of the 3xBF16 method, as float64 matrices.

    Returns the exact value ``hi_a@hi_b + hi_a@lo_b + lo_a@hi_b`` factors:
    (Ahi, Alo, Bhi, Blo) as float64 so the caller can form the sum with the
    FP64 oracle GEMM.
    """
    ah, al = split_bf16(A)
    bh, bl = split_bf16(B)
    f = lambda b: bf16_to_f32(b).astype(np.float64)
    return f(ah), f(al), f(bh), f(bl)


# ---------------------------------------------------------------- error metric
def rel_frobenius(C, C_ref):
    """||C - C_ref||_F / ||C_ref||_F in float64 (0/0 -> 0, x/0 -> inf)."""
    C = np.asarray(C, dtype=np.float64)
    C_ref = np.asarray(C_ref, dtype=np.float64)
    num = np.linalg.norm((C - C_ref).ravel())
    den = np.linalg.norm(C_ref.ravel())
    if den == 0:
        return 0.0 if num == 0 else float("inf")
    return float(num / den)
