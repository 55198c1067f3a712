"""Shared helpers of the test-suite: storage-type rounding, tolerances, and the
scaled magnitudes used to bound rounding differences (|y - y_ref| <= tol * M),
and the tighter check of a low-precision output against the exact result
rounded once to its format."""
import numpy as np

from paper_2007_07539_gb300 import mg

# Tolerance on |gpu - oracle| relative to the componentwise scaled magnitude M.
TOL = {mg.FP64: 1e-12, mg.FP32: 1e-5, mg.FP16: 5e-3, mg.BF16: 5e-3}
NAME = {mg.FP64: "fp64", mg.FP32: "fp32", mg.FP16: "fp16", mg.BF16: "bf16"}


def to_storage(x: np.ndarray, prec: int):
    """Round FP64 values to the storage type (round to nearest even).
    Returns (host buffer for mg_level_write, the rounded values as FP64)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    if prec == mg.FP64:
        return x, x.copy()
    if prec == mg.FP32:
        b = x.astype(np.float32)
        return b, b.astype(np.float64)
    if prec == mg.FP16:
        b = x.astype(np.float16)
        return b, b.astype(np.float64)
    import torch
    t = torch.from_numpy(x).to(torch.bfloat16).contiguous()
    return t, t.to(torch.float64).numpy()


def empty_storage(shape, prec: int):
    if prec == mg.FP64:
        return np.zeros(shape, np.float64)
    if prec == mg.FP32:
        return np.zeros(shape, np.float32)
    if prec == mg.FP16:
        return np.zeros(shape, np.float16)
    import torch
    return torch.zeros(shape, dtype=torch.bfloat16)


def as_f64(buf) -> np.ndarray:
    if hasattr(buf, "to"):
        import torch
        return buf.to(torch.float64).numpy()
    return np.asarray(buf, dtype=np.float64)


def check_close(got, ref, mag, prec, what=""):
    """Asserts |got - ref| <= TOL[prec] * mag elementwise (mag floored at a tiny value)."""
    got, ref, mag = (np.asarray(a, dtype=np.float64) for a in (got, ref, mag))
    assert got.shape == ref.shape, (got.shape, ref.shape)
    assert np.all(np.isfinite(got)), f"{what}: non-finite output"
    bound = TOL[prec] * np.maximum(mag, 1e-300)
    err = np.abs(got - ref)
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError(f"{what} [{NAME[prec]}]: {bad.sum()} of {bad.size} points exceed tol; worst at {i}: "
                             f"got {got[i]!r} ref {ref[i]!r} mag {mag[i]!r} ratio {(err / bound)[i]:.3g}")


# significand bits (leading bit included) and least normal exponent of the storage formats
_FMT = {mg.FP32: (24, -126), mg.FP16: (11, -14), mg.BF16: (8, -126)}


def ulp(x, prec) -> np.ndarray:
    """Spacing of the storage format at |x|: 2^(e - p + 1) in the binade [2^e, 2^(e+1)),
    the subnormal spacing 2^(emin - p + 1) below the least normal 2^emin."""
    p, emin = _FMT[prec]
    a = np.abs(np.asarray(x, dtype=np.float64))
    _, e = np.frexp(a)  # a = f 2^e, f in [1/2, 1)
    e = np.where(a > 0, np.maximum(e - 1, emin), emin)
    return np.ldexp(1.0, e - p + 1)


def check_rounded(oracle, got, ref, mag, prec, what="", k=32):
    """A low-precision output against the exact (FP64) result rounded once to its
    format by the oracle:  |got - round(ref)| <= ulp(max(|got|, |round(ref)|)) + k 2^-24 mag.
    The kernel computes v in FP32 with |v - ref| <= k 2^-24 mag and stores round(v);
    each of the two roundings moves a value by at most half a spacing, so the bound
    holds for a kernel that rounds once per stored value (Sec. 6, FP32 arithmetic
    inside FP16/BF16 levels).  Applied to FP16 and BF16 outputs, where the
    k 2^-24 mag term is far below one spacing; FP32 and FP64 outputs are
    held to check_close only."""
    if prec not in (mg.FP16, mg.BF16):
        return
    code = {mg.FP16: oracle.FP16, mg.BF16: oracle.BF16}[prec]
    got, ref, mag = (np.asarray(a, dtype=np.float64) for a in (got, ref, mag))
    rr = oracle.round_to(code, ref)
    bound = ulp(np.maximum(np.abs(got), np.abs(rr)), prec) + k * 2.0**-24 * mag
    err = np.abs(got - rr)
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError(f"{what} [{NAME[prec]}]: {bad.sum()} of {bad.size} points beyond one rounding; "
                             f"worst at {i}: got {got[i]!r} rounded ref {rr[i]!r} ref {ref[i]!r} mag {mag[i]!r}")
