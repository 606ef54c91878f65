"""Bit-exact check of the library's integer-only FP64 <-> FP32 conversions (the MIXED path's
narrow, split_df and widen, which keep conversions off the FP64 unit), built for the host with
g++, against IEEE-754 conversions in numpy: narrow(d) is the float nearest to d, ties to even;
split_df gives that float and the float nearest to the remainder; widen is exact. Documented
exceptions: magnitudes below the FP32 normal range give signed zero (numpy gives subnormals),
and so does widen of an FP32 subnormal; the low part is zero for |d| < 2^-74 (its unit would be
subnormal). No GPU."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from tests.test_host_device_math import FLAGS, HOST

F32_MIN_NORMAL = float(np.finfo(np.float32).tiny)


def _doubles(rng, n):
    """Doubles across the FP32 range and beyond, exact FP32 ties, and special values."""
    e = rng.integers(-140, 140, n)
    d = rng.uniform(1.0, 2.0, n) * np.exp2(e.astype(np.float64)) * rng.choice([-1.0, 1.0], n)
    # exact ties: a float plus half its ulp (both parities of the last mantissa bit)
    f = rng.uniform(1.0, 2.0, n // 4).astype(np.float32) * np.exp2(rng.integers(-100, 100, n // 4)).astype(np.float32)
    ulp = np.spacing(f).astype(np.float64)
    ties = f.astype(np.float64) + 0.5 * ulp
    specials = np.array([0.0, -0.0, np.inf, -np.inf, 1.0, -1.0, float(np.finfo(np.float32).max),
                         float(np.finfo(np.float32).max) * (1 + 2 ** -25), float(np.finfo(np.float32).max) * (1 + 2 ** -23),
                         F32_MIN_NORMAL, -F32_MIN_NORMAL, F32_MIN_NORMAL * (1 - 2 ** -30), 2.0 ** 127, 2.0 ** 128,
                         1.0 + 2 ** -24, 1.0 + 2 ** -24 + 2 ** -50, 1.0 - 2 ** -25, 3.0 * 2 ** -150])
    return np.concatenate([d, ties, specials])


@pytest.fixture(scope="module")
def converted(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path_factory.mktemp("conversions") / "conversions")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "conversions.cpp"), "-o", exe], capture_output=True,
                           text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    rng = np.random.default_rng(9)
    d = _doubles(rng, 20000)
    f = np.concatenate([rng.standard_normal(d.size - 6).astype(np.float32) * np.exp2(rng.integers(-120, 120, d.size - 6)).astype(np.float32),
                        np.array([0.0, -0.0, np.inf, -np.inf, 1e-40, -3e-39], dtype=np.float32)])
    db = d.view(np.uint64)
    fb = f.view(np.uint32)
    stdin = f"{d.size}\n" + "\n".join(f"{int(a):016x} {int(b):08x}" for a, b in zip(db, fb)) + "\n"
    run = subprocess.run([exe], input=stdin, capture_output=True, text=True, timeout=120)
    assert run.returncode == 0, run.stderr[-2000:]
    rows = [line.split() for line in run.stdout.splitlines()]
    assert len(rows) == d.size
    narrow = np.array([int(r[0], 16) for r in rows], dtype=np.uint32).view(np.float32)
    hi = np.array([int(r[1], 16) for r in rows], dtype=np.uint32).view(np.float32)
    lo = np.array([int(r[2], 16) for r in rows], dtype=np.uint32).view(np.float32)
    wide = np.array([int(r[3], 16) for r in rows], dtype=np.uint64).view(np.float64)
    return d, f, narrow, hi, lo, wide


def _same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32 if a.dtype == np.float32 else np.uint64),
                          np.asarray(b).view(np.uint32 if b.dtype == np.float32 else np.uint64))


def test_narrow_is_round_to_nearest_even(converted):
    d, _, narrow, hi, _, _ = converted
    with np.errstate(over="ignore"):
        ref = d.astype(np.float32)   # IEEE round to nearest, ties to even; overflow to infinity
    tiny = np.abs(d) < F32_MIN_NORMAL
    ref[tiny] = np.copysign(np.float32(0.0), d[tiny]).astype(np.float32)
    assert _same_bits(narrow, ref)
    assert _same_bits(hi, ref)


def test_split_low_part(converted):
    d, _, _, hi, lo, _ = converted
    fin = np.isfinite(hi) & (hi != 0)
    rem = d[fin] - hi[fin].astype(np.float64)          # exact in FP64
    ref = rem.astype(np.float32)
    ref[np.abs(d[fin]) < 2.0 ** -74] = np.float32(0.0)   # the remainder's unit is below the normal range
    got = lo[fin].copy()
    got[got == 0] = np.float32(0.0)                     # compare zeros without their sign
    ref[ref == 0] = np.float32(0.0)
    assert _same_bits(got, ref)
    # hi + lo carries d to about 2^-48 relative where the low part is representable
    ok = np.abs(d[fin]) >= 2.0 ** -74
    carried = hi[fin][ok].astype(np.float64) + lo[fin][ok].astype(np.float64)
    assert np.all(np.abs(carried - d[fin][ok]) <= 2.0 ** -47 * np.abs(d[fin][ok]))
    assert np.all(lo[~fin] == 0)


def test_widen_is_exact(converted):
    _, f, _, _, _, wide = converted
    ref = f.astype(np.float64)
    sub = (np.abs(f) < F32_MIN_NORMAL) & (f != 0)
    ref[sub] = np.copysign(0.0, f[sub].astype(np.float64))
    assert _same_bits(wide, ref)


def test_device_nesterov_scalar_is_the_oracles(tmp_path):
    """nesterov_next (Eq. nesterov_scalar on the device, each operation rounded separately) gives
    the oracle's s^(k) bit for bit over 5,000 iterations, so that a run whose momentum reset keeps
    s on the device takes the same extrapolation ratios as the host-computed table."""
    from oracle import daba_oracle as O
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "scalars")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "scalars.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    n = 5000
    run = subprocess.run([exe], input=f"{n}\n", capture_output=True, text=True, timeout=60)
    assert run.returncode == 0
    dev = np.array([int(x, 16) for x in run.stdout.split()], dtype=np.uint64).view(np.float64)
    ref = [1.0]
    for _ in range(n):
        ref.append(float(O.nesterov(ref[-1])[0]))
    assert _same_bits(dev, np.array(ref))


def test_double_float_addition_against_exact_sums(tmp_path):
    """df_add, the (hi, lo) FP32-pair update of the MIXED landmark state: for seeded pairs with
    |lo| <= ulp(hi)/2 and steps from 1e-9 |hi| to 10 |hi| (both signs, exact cancellation, zero
    and steps below ulp(lo) included), the new pair sums to hi + lo + x within 2^-46 of the
    larger of |hi| and |x| (exact rational arithmetic), and its low part is at most half an ulp
    of its high part."""
    import struct
    from fractions import Fraction
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "df_add")
    build = subprocess.run([gxx, *FLAGS, os.path.join(HOST, "df_add.cpp"), "-o", exe], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr[-4000:]
    rng = np.random.default_rng(17)
    n = 4000
    hi = (rng.uniform(-100, 100, n) * 10.0 ** rng.uniform(-3, 2, n)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float32)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    x = (hi.astype(np.float64) * rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-9, 1, n)).astype(np.float32)
    x[0::50] = -hi[0::50]                        # exact cancellation of the high part
    x[1::50] = 0.0
    x[2::50] = (lo[2::50] * np.float32(1e-3))    # below the low part's ulp
    bits = lambda a: a.view(np.uint32)
    stdin = f"{n}\n" + "\n".join(f"{h:08x} {l:08x} {v:08x}" for h, l, v in zip(bits(hi), bits(lo), bits(x))) + "\n"
    run = subprocess.run([exe], input=stdin, capture_output=True, text=True, timeout=60)
    assert run.returncode == 0, run.stderr[-2000:]
    out = np.array([[int(w, 16) for w in line.split()] for line in run.stdout.splitlines()], dtype=np.uint32)
    h2, l2 = out[:, 0].view(np.float32), out[:, 1].view(np.float32)
    f = lambda v: Fraction(struct.unpack("<f", struct.pack("<f", float(v)))[0])
    for i in range(n):
        exact = f(hi[i]) + f(lo[i]) + f(x[i])
        got = f(h2[i]) + f(l2[i])
        bound = Fraction(2) ** -46 * max(abs(f(hi[i])), abs(f(x[i])), Fraction(1, 2 ** 100))
        assert abs(got - exact) <= bound, (i, float(got - exact), float(bound))
        assert abs(float(l2[i])) <= 0.5 * float(np.spacing(np.abs(h2[i]))), i
