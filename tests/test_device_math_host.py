"""The library's exact-arithmetic helpers (csrc/gs_device.cuh), built for the
host with g++, against Python Fractions.  On the device these form every sum
and quotient of the GS_FP64 path; here they are checked one by one:
  * to_fixed: a float64 as a two's-complement integer in units of 2^L
    (truncated toward zero; inexact / out-of-window flags);
  * round_fixed: V * 2^L rounded to the nearest float64, ties to even,
    subnormals included;
  * round_to_double: the same rounding kept in units of 2^L (equal to
    to_fixed(round_fixed(V, L), L));
  * div_round: the exact quotient V * 2^L / D rounded once, ties to even,
    or the inexact flag where the quotient has too few bits to round (its
    documented limit);
  * the exact float32 -> float64 widening of the bit patterns;
  * key_index: the cell of a value by a float guess corrected against the
    exact face table (the device's floor(x / h))."""
from __future__ import annotations

import math
import os
import random
import shutil
import struct
import subprocess
from fractions import Fraction as Fr

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M128 = (1 << 128) - 1


@pytest.fixture(scope="module")
def dm(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("devmath")
    # the header includes <cuda_runtime.h>; the host build needs none of it
    (d / "cuda_runtime.h").write_text("")
    exe = str(d / "device_math_host")
    b = subprocess.run([gxx, "-std=c++17", "-O2", "-Wno-unknown-pragmas", "-I", str(d),
                        "-o", exe, os.path.join(ROOT, "tests", "device_math_host_driver.cpp")],
                       capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-3000:]

    def ask(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                           text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-1000:]
        out = r.stdout.strip().splitlines()
        assert len(out) == len(lines)
        return out
    return ask


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def from_bits(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def split(v: int) -> str:
    v &= M128
    return f"{v >> 64:x} {v & ((1 << 64) - 1):x}"


def signed(hi: str, lo: str) -> int:
    v = (int(hi, 16) << 64) | int(lo, 16)
    return v - (1 << 128) if v >> 127 else v


def rn(q: Fr) -> float:
    return float(q)  # Python rounds a Fraction correctly (ties to even, subnormals)


def _values(rng, n):
    """Signed integers of every width up to 125 bits, and tie patterns."""
    out = []
    for _ in range(n):
        w = rng.randint(1, 125)
        v = rng.getrandbits(w) | (1 << (w - 1))
        out.append(v if rng.random() < 0.5 else -v)
    for w in (54, 60, 80, 120):  # exact ties at the 53-bit boundary, odd and even
        for last in (0, 1):
            top = (1 << 52) | rng.getrandbits(51) << 1 | last
            v = (2 * top + 1) << (w - 54)
            out += [v, -v]
    return out


LS = [-1100, -1075, -300, -64, -20, 0, 17]


def test_to_fixed(dm):
    rng = random.Random(1)
    cases = []
    for _ in range(400):
        x = rng.uniform(-1, 1) * 2.0 ** rng.randint(-1080, 120)
        cases.append((x, rng.choice(LS)))
    cases += [(0.0, 0), (-0.0, 5), (5e-324, -1074), (5e-324, -1000), (2.0 ** 125, 0),
              (2.0 ** 126, 0), (-(2.0 ** 200), 70)]
    out = dm([f"T {bits(x):x} {L}" for x, L in cases])
    for (x, L), line in zip(cases, out):
        hi, lo, inexact, err = line.split()
        q = Fr(x) / Fr(2) ** L
        if abs(q) >= 2 ** 126:
            assert err == "1", (x, L)
            continue
        assert err == "0", (x, L)
        t = math.trunc(q)  # toward zero
        assert signed(hi, lo) == t, (x, L)
        assert inexact == ("1" if q != t else "0"), (x, L)


def test_round_fixed_and_round_to_double(dm):
    rng = random.Random(2)
    cases = [(v, rng.choice(LS)) for v in _values(rng, 500)]
    out_r = dm([f"R {split(v)} {L}" for v, L in cases])
    out_q = dm([f"Q {split(v)} {L}" for v, L in cases])
    for (v, L), r, q in zip(cases, out_r, out_q):
        want = rn(Fr(v) * Fr(2) ** L)
        assert int(r, 16) == bits(want) or (want == 0 and from_bits(int(r, 16)) == 0), (v, L)
        hi, lo, err = q.split()
        back = Fr(want) / Fr(2) ** L
        assert back.denominator == 1
        assert signed(hi, lo) == back.numerator, (v, L)
        assert err == ("1" if abs(back) >= 2 ** 126 else "0")


def test_div_round(dm):
    rng = random.Random(3)
    cases = []
    for v in _values(rng, 400):
        D = rng.choice([1, 2, 3, 7, 1 << 31, (1 << 32) - 1, rng.randint(1, (1 << 32) - 1),
                        rng.randint(1, 1000)])
        cases.append((v, D, rng.choice(LS)))
    for _ in range(100):  # quotients that are exact ties
        D = rng.randint(1, 1 << 20)
        top = (1 << 52) | rng.getrandbits(52)
        X = (2 * top + 1) << rng.randint(0, 40)
        if X * D < 1 << 125:
            cases.append((X * D * rng.choice([1, -1]), D, rng.choice(LS)))
    cases += [(-38, 3986530705, 17), (1, (1 << 32) - 1, 0)]  # quotients of few bits
    out = dm([f"V {split(v)} {D} {L}" for v, D, L in cases])
    flagged = 0
    for (v, D, L), line in zip(cases, out):
        b, inexact = line.split()
        want = rn(Fr(v) * Fr(2) ** L / D)
        got = from_bits(int(b, 16))
        Q, R = divmod(abs(v) << 64, D)  # the 64 fraction bits the division forms
        if inexact == "1":
            # the documented limit: the quotient has at most 53 bits there and
            # a nonzero remainder, so the rounding is unknown and flagged
            assert Q.bit_length() <= 53 and R != 0, (v, D, L)
            flagged += 1
            continue
        assert got == want and math.copysign(1, got) == math.copysign(1, want) or \
            (want == 0 and got == 0), (v, D, L, got, want)
    assert flagged >= 2 and flagged < len(cases) // 10


def test_float32_widening(dm):
    rng = random.Random(4)
    fs = [0, 0x80000000, 1, 0x807FFFFF, 0x00400000, 0x3F800000, 0x7F7FFFFF, 0xFF7FFFFF]
    fs += [rng.getrandbits(32) for _ in range(500)]
    fs = [f for f in fs if (f >> 23) & 0xFF != 0xFF]  # finite inputs only
    out = dm([f"W {f:x}" for f in fs])
    for f, line in zip(fs, out):
        x = struct.unpack("<f", struct.pack("<I", f))[0]  # exact in a Python float
        assert int(line, 16) == bits(x), hex(f)


def test_u32_to_double(dm):
    # the image features' channel bytes and the like, converted with integer
    # instructions: every 16-bit value, the powers of two and their
    # neighbours, and random 32-bit values, against Python's exact float()
    rng = random.Random(6)
    vs = list(range(1 << 16))
    vs += [(1 << k) + o for k in range(16, 32) for o in (-1, 0, 1)] + [0xFFFFFFFF]
    vs += [rng.getrandbits(32) for _ in range(2000)]
    out = dm([f"I {v:x}" for v in vs])
    for v, line in zip(vs, out):
        assert int(line, 16) == bits(float(v)), hex(v)


def test_key_index_is_floor(dm):
    rng = random.Random(5)
    cases = []
    for h in (0.1, 1.0 / 3.0, 12.0, 1e-3, 7.5e5, 0.75, 2.0 ** -20, 16.0):
        for _ in range(120):
            span = rng.choice([1, 2, 3, rng.randint(1, 5000)])
            kmin = rng.randint(-10 ** 6, 10 ** 6)
            q = kmin + rng.randrange(span)
            lo = Fr(q) * Fr(h)
            f = float(lo)
            if Fr(f) < lo:
                f = math.nextafter(f, math.inf)  # the face of cell q
            kind = rng.randrange(3)
            if kind == 0:
                x = f
            elif kind == 1:
                x = float(lo + Fr(h) * Fr(rng.random()))
            else:
                x = math.nextafter(f, -math.inf) if q > kmin else f
            cases.append((h, kmin, span, x))
    out = dm([f"K {h.hex()} {kmin} {span} {x.hex()}" for h, kmin, span, x in cases])
    for (h, kmin, span, x), got in zip(cases, out):
        want = math.floor(Fr(x) / Fr(h)) - kmin
        want = min(max(want, 0), span - 1)  # outside the table: clamped
        assert int(got) == want, (h, kmin, span, x)


def _home(key: int, buckets: int) -> int:
    b = buckets.bit_length() - 1  # buckets is a power of two
    return 0 if b == 0 else ((key * 0x9E3779B97F4A7C15) % 2 ** 64) >> (64 - b)


def test_hash_table_insert_and_lookup(dm):
    # one thread: every distinct key gets its own slot within the probe limit
    # of its home bucket (Fibonacci hashing, four slots a bucket); a repeated
    # insert returns the same slot without winning; lookups find every stored
    # key and no absent one; an insert that finds no free slot within the
    # limit returns no slot and sets kErrTableFull (never at load <= 1/2)
    rng = random.Random(6)
    cases = []
    for cap in (4, 16, 64, 1024, 4096):
        for load in (0.25, 0.5, 0.9, 1.0, 1.3):
            n = int(cap * load)
            keys = [rng.getrandbits(63) for _ in range(n)]
            keys += rng.sample(keys, min(len(keys), 5))  # repeats
            absent = [rng.getrandbits(63) | (1 << 62) for _ in range(10)]
            cases.append((cap, keys, keys[:50] + absent))
    lines = [f"H {cap} {len(ins)} " + " ".join(f"{k:x}" for k in ins) + f" {len(look)} "
             + " ".join(f"{k:x}" for k in look) for cap, ins, look in cases]
    out = dm(lines)
    for (cap, ins, look), line in zip(cases, out):
        f = line.split()
        slots = [int(x, 16) for x in f[0:2 * len(ins):2]]
        wons = [int(x) for x in f[1:2 * len(ins):2]]
        found = [int(x, 16) for x in f[2 * len(ins):2 * len(ins) + len(look)]]
        err = int(f[-1])
        buckets = cap // 4
        where = {}
        failed = False
        for k, sl, won in zip(ins, slots, wons):
            if sl == 0xFFFFFFFF:  # no free slot within the probe limit
                failed = True
                assert won == 0 and k not in where
                continue
            assert sl < cap
            if k in where:
                assert sl == where[k] and won == 0
            else:
                assert won == 1 and sl not in where.values()
                where[k] = sl
                dist = (sl // 4 - _home(k, buckets)) % buckets
                assert dist < min(buckets, 128)  # within the probe limit
        assert bool(err & 1) == failed
        if len(set(ins)) > cap:
            assert failed
        if len(set(ins)) <= cap // 2:  # the loads the library uses
            assert not failed
        for k, sl in zip(look, found):
            assert sl == where.get(k, 0xFFFFFFFF), (cap, k)
