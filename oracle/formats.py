"""Number formats, unit roundoffs and rounding for the oracle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Unit roundoffs are those of Table 3 of the paper (fp16 2^-11, fp32 2^-24,
fp64 2^-53, quad 2^-113); bfloat16 (mentioned in Sec. 2.2 and Sec. 4 as a
possible non-IEEE format) has 8 significant bits, u = 2^-8.  The paper's
quad residual precision is stood in for by double-double (dd), whose unit
roundoff 2^-106 is exactly u^2 for u = fp64.

Every quantity of a format below fp64 is held in a float32 or float64 numpy
array whose values are exactly representable in that format.  Rounding is
IEEE round-to-nearest-even with gradual underflow and overflow to +-Inf
(reading: the paper only says "rounding").  16-bit formats are always
rounded from a float32 value, so fl16(x) for a float64 x means
fl16(fl32(x)).

Double-double numbers are pairs (hi, lo) of float64 arrays with
|lo| <= ulp(hi)/2.  The error-free transformations are Knuth's TwoSum,
Dekker's FastTwoSum and Dekker's TwoProduct with Veltkamp splitting
(no fused multiply-add is needed); dd addition is the accurate
("IEEE-style") addition of Hida, Li and Bailey's QD library, restated from
its published description.
"""

import numpy as np

# Format codes; they equal the codes of the library's C interface so that a
# test can pass one value to both sides.
BF16, FP16, FP32, FP64, DD = 1, 2, 3, 4, 5
NAMES = {BF16: "bf16", FP16: "fp16", FP32: "fp32", FP64: "fp64", DD: "dd"}

# Unit roundoff u = 2^-p (Table 3; bf16 and dd as stated above).
UNIT_ROUNDOFF = {
    BF16: 2.0 ** -8,
    FP16: 2.0 ** -11,
    FP32: 2.0 ** -24,
    FP64: 2.0 ** -53,
    DD: 2.0 ** -106,
}
# Largest finite value, used by the squeezing scaling.
XMAX = {
    BF16: float(np.float32(3.3895313892515355e38)),
    FP16: 65504.0,
    FP32: float(np.finfo(np.float32).max),
    FP64: float(np.finfo(np.float64).max),
}


def u_of(fmt):
    return UNIT_ROUNDOFF[fmt]


def next_uf(fmt):
    """Next factorisation precision when Algorithm 4 sets u_f = u_f^2.

    Reading: "u_f^2" is taken as the least IEEE format whose unit roundoff is
    at most u_f^2: half/bfloat16 -> single -> double (Sec. 2, example after
    Algorithm 4).  Beyond double there is no next format (None)."""
    return {BF16: FP32, FP16: FP32, FP32: FP64, FP64: None}[fmt]


def square_of(fmt):
    """The precision u^2 used by GMRES-IR's operator and enforced for u_r."""
    return {FP32: FP64, FP64: DD}[fmt]


# ---------------------------------------------------------------- rounding

def fl32(x):
    """Round to IEEE single (numpy's float64->float32 cast is RNE)."""
    return np.asarray(x, dtype=np.float64).astype(np.float32)


def fl16(x):
    """Round to IEEE half; float64 input is first rounded to single."""
    x32 = np.asarray(x).astype(np.float32) if np.asarray(x).dtype != np.float32 else np.asarray(x)
    with np.errstate(over="ignore"):
        return x32.astype(np.float16).astype(np.float32)


def flbf16(x):
    """Round to bfloat16 (8 significant bits, fp32 exponent range), RNE.

    Works on the float32 bit pattern: add 0x7FFF plus the lowest kept bit,
    then clear the 16 dropped bits.  A carry into the exponent field gives the
    next binade or +-Inf, as IEEE rounding does.  NaN stays NaN."""
    x32 = np.array(np.asarray(x).astype(np.float32), dtype=np.float32, copy=True)
    bits = x32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)).astype(np.uint32)
    out = rounded.view(np.float32)
    nan = np.isnan(x32)
    if np.any(nan):
        out = np.where(nan, np.float32(np.nan), out)
    return out


def chop(x, fmt):
    """One IEEE round-to-nearest-even rounding of float64 values to ``fmt``,
    with no fp32 step in between: the rounding of the paper's simulated low
    precisions (Sec. 3 simulates half precision by rounding every result of
    a double-precision operation to half).  Gradual underflow; overflow to
    +-Inf.  Returns float64.

    fp16: numpy's float64 -> float16 conversion (one correct rounding).
    bf16 (8 significant bits, exponent range of fp32): in the normal range
    the float64 significand is rounded to 8 bits with integer arithmetic on
    its bit pattern; below 2^-126 the value is rounded to a multiple of the
    subnormal spacing 2^-133."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(all="ignore"):
        if fmt == FP64:
            return x.copy()
        if fmt == FP32:
            return x.astype(np.float32).astype(np.float64)
        if fmt == FP16:
            return x.astype(np.float16).astype(np.float64)
        if fmt == BF16:
            bits = np.ascontiguousarray(x).view(np.uint64)
            drop = np.uint64(52 - 7)
            lsb = (bits >> drop) & np.uint64(1)
            half = np.uint64((1 << 44) - 1)
            mask = ~np.uint64((1 << 45) - 1)
            r = ((bits + half + lsb) & mask).view(np.float64).reshape(x.shape)
            r = np.where(np.isfinite(x), r, x)
            tiny = np.abs(x) < 2.0 ** -126
            r = np.where(tiny, np.round(x * 2.0 ** 133) * 2.0 ** -133, r)
            r = np.where(np.abs(r) > XMAX[BF16], np.copysign(np.inf, x), r)
            return r
    raise ValueError(f"no single-word rounding for format {fmt}")


def fl(x, fmt):
    """Round x (float32/float64 values) to format ``fmt``.

    Returns float32 for bf16/fp16/fp32 and float64 for fp64."""
    if fmt == FP64:
        return np.asarray(x, dtype=np.float64)
    if fmt == FP32:
        return fl32(x)
    if fmt == FP16:
        return fl16(x)
    if fmt == BF16:
        return flbf16(x)
    raise ValueError(f"no single-word rounding for format {fmt}")


def arith_dtype(fmt):
    """numpy dtype in which a format's own arithmetic is carried out."""
    return np.float64 if fmt == FP64 else np.float32


# ------------------------------------------------------- double-double

_SPLITTER = 134217729.0  # 2^27 + 1 (Veltkamp)


def two_sum(a, b):
    """Knuth TwoSum: s + e == a + b exactly, s = fl(a + b)."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def fast_two_sum(a, b):
    """Dekker FastTwoSum, valid when |a| >= |b| (or a == 0)."""
    s = a + b
    e = b - (s - a)
    return s, e


def split(a):
    t = _SPLITTER * a
    hi = t - (t - a)
    lo = a - hi
    return hi, lo


def two_prod(a, b):
    """Dekker TwoProduct: p + e == a * b exactly, p = fl(a * b)."""
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def dd(hi, lo=None):
    hi = np.asarray(hi, dtype=np.float64)
    lo = np.zeros_like(hi) if lo is None else np.asarray(lo, dtype=np.float64)
    return hi, lo


def dd_add(a, b):
    """Accurate dd + dd (QD 'ieee_add')."""
    s, e = two_sum(a[0], b[0])
    t, f = two_sum(a[1], b[1])
    e = e + t
    s, e = fast_two_sum(s, e)
    e = e + f
    return fast_two_sum(s, e)


def dd_neg(a):
    return -a[0], -a[1]


def dd_sub(a, b):
    return dd_add(a, dd_neg(b))


def dd_mul_d(a, d):
    """dd * double."""
    p, e = two_prod(a[0], d)
    e = e + a[1] * d
    return fast_two_sum(p, e)


def dd_mul(a, b):
    p, e = two_prod(a[0], b[0])
    e = e + (a[0] * b[1] + a[1] * b[0])
    return fast_two_sum(p, e)


def dd_div(a, b):
    """dd / dd by three rounds of long division (QD 'accurate_div')."""
    q1 = a[0] / b[0]
    r = dd_sub(a, dd_mul_d(b, q1))
    q2 = r[0] / b[0]
    r = dd_sub(r, dd_mul_d(b, q2))
    q3 = r[0] / b[0]
    q = fast_two_sum(q1, q2)
    return dd_add(q, dd(q3))


def dd_div_d(a, d):
    return dd_div(a, dd(d))


def dd_sum_pairwise(terms, axis=-1):
    """Sum dd terms along ``axis`` by a balanced pairwise tree of dd_add."""
    hi, lo = np.moveaxis(terms[0], axis, -1), np.moveaxis(terms[1], axis, -1)
    if hi.shape[-1] == 0:
        z = np.zeros(hi.shape[:-1])
        return z, z.copy()
    while hi.shape[-1] > 1:
        if hi.shape[-1] % 2:
            pad = [(0, 0)] * (hi.ndim - 1) + [(0, 1)]
            hi = np.pad(hi, pad)
            lo = np.pad(lo, pad)
        hi, lo = dd_add((hi[..., 0::2], lo[..., 0::2]), (hi[..., 1::2], lo[..., 1::2]))
    return hi[..., 0], lo[..., 0]


def dd_to_fp64(a):
    """Round a normalised dd to fp64: the high word (|lo| <= ulp(hi)/2)."""
    return np.asarray(a[0] + a[1], dtype=np.float64)


def dd_to_fp32(a):
    """Round a normalised dd to fp32 correctly (one rounding of hi + lo).

    fl32(hi) is already the answer unless hi lies exactly halfway between
    two fp32 neighbours; then the sign of lo decides (a nonzero lo moves the
    exact value off the tie, towards the neighbour on its side)."""
    hi = np.asarray(a[0], dtype=np.float64)
    lo = np.asarray(a[1], dtype=np.float64)
    with np.errstate(all="ignore"):
        r = hi.astype(np.float32)
        r64 = r.astype(np.float64)
        d = hi - r64  # exact: |d| <= half an fp32 ulp of hi
        other = np.nextafter(r, (r64 + 2.0 * d).astype(np.float32))
        tie = np.isfinite(r64) & (d != 0) & (other.astype(np.float64) - r64 == 2.0 * d)
        away = tie & (lo != 0) & (np.sign(lo) == np.sign(d))
        return np.where(away, other, r)


def dd_abs_max(a):
    """max_i |a_i| of a dd vector, returned as fp64 (the high word of the max)."""
    hi = np.abs(a[0])
    if hi.size == 0:
        return 0.0
    return float(np.max(np.abs(dd_to_fp64(a))))
