"""The library's planner (csrc/gs_planner.cuh), built for the host with g++,
against exact arithmetic.  The same functions run on the device (the
key-range kernel) and decide every cell key of Sec. 2.1 i, so they are
checked here on the CPU:
  * plan_floor_div(x, h) = floor of the exact quotient x / h (Python
    Fractions), on random values and on both sides of exact cell faces;
  * plan_face(q, h) = the least double >= q h;
  * plan_ord_of orders doubles as their values (-0 as +0);
  * plan_finish / plan_probe: the packed-key layout (axis 0 most significant,
    each axis span + 1 values wide, the instance field above) and the 3^d
    neighbour offsets (axis 0 the slowest digit);
  * plan_from_range: the whole plan from a key range, and its refusals."""
from __future__ import annotations

import math
import os
import random
import shutil
import subprocess
from fractions import Fraction as Fr

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("planner") / "planner_host")
    b = subprocess.run([gxx, "-std=c++17", "-O2", "-ffp-contract=off", "-o", exe,
                        os.path.join(ROOT, "tests", "planner_host_driver.cpp")],
                       capture_output=True, text=True)
    assert b.returncode == 0, b.stderr[-2000:]

    def ask(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True,
                           text=True, timeout=300)
        assert r.returncode == 0, r.stderr[-1000:]
        out = r.stdout.strip().splitlines()
        assert len(out) == len(lines)
        return out
    return ask


def least_double_at_least(v: Fr) -> float:
    t = float(v)  # nearest
    if Fr(t) < v:
        t = math.nextafter(t, math.inf)
    return t


HS = [0.1, 1.0 / 3.0, 12.0, 1e-3, 7.5e5, 1.0, 0.75, 2.0 ** -20, 16.0, 4.0]


def test_floor_div_is_exact(planner):
    rng = random.Random(2206)
    cases = []
    for h in HS:
        for _ in range(150):
            x = rng.uniform(-1, 1) * 10.0 ** rng.randint(-3, 9) * h
            cases.append((x, h))
        for _ in range(60):  # both sides of an exact face
            q = rng.randint(-10 ** 6, 10 ** 6)
            f = least_double_at_least(Fr(q) * Fr(h))
            cases += [(f, h), (math.nextafter(f, -math.inf), h)]
    out = planner([f"F {x.hex()} {h.hex()}" for x, h in cases])
    for (x, h), got in zip(cases, out):
        assert int(got) == math.floor(Fr(x) / Fr(h)), (x, h)


def test_face_is_least_double_above(planner):
    rng = random.Random(7)
    cases = [(rng.randint(-2 ** 40, 2 ** 40), h) for h in HS for _ in range(100)]
    cases += [(q, h) for h in HS for q in (-3, -1, 0, 1, 2, 3)]
    out = planner([f"A {q} {h.hex()}" for q, h in cases])
    for (q, h), got in zip(cases, out):
        assert float.fromhex(got) == least_double_at_least(Fr(q) * Fr(h)), (q, h)


def test_order_codes_follow_values(planner):
    rng = random.Random(11)
    xs = [0.0, -0.0, 5e-324, -5e-324, 1.0, -1.0, 1e308, -1e308, 2.2250738585072014e-308]
    xs += [rng.uniform(-1, 1) * 10.0 ** rng.randint(-300, 300) for _ in range(400)]
    out = [int(v) for v in planner([f"O {x.hex()}" for x in xs])]
    code = dict(zip(xs, out))
    assert code[0.0] == code[-0.0] == 0
    order = sorted(set(xs))
    codes = [code[x] for x in order]
    assert all(a < b for a, b in zip(codes, codes[1:]))


def test_packed_key_layout_and_probes(planner):
    rng = random.Random(5)
    cases = []
    for _ in range(60):
        d = rng.randint(1, 8)
        B = rng.choice([1, 1, 2, 64, 1000])
        spans = [rng.choice([1, 2, 3, rng.randint(1, 300), rng.randint(1, 5000)])
                 for _ in range(d)]
        cases.append((d, B, spans))
    cases.append((8, 1, [1000] * 8))  # 80 bits: refused
    out = planner([f"L {d} {B} " + " ".join(map(str, s)) for d, B, s in cases])
    for (d, B, spans), line in zip(cases, out):
        f = line.split()
        width = [(s + 1).bit_length() for s in spans]
        total = sum(width) + ((B - 1).bit_length() if B > 1 else 0)
        assert int(f[1]) == total
        if total > 63:
            assert int(f[0]) == 4  # kPlanBits
            continue
        assert int(f[0]) == 0
        off = [sum(width[a + 1:]) for a in range(d)]  # axis 0 most significant
        got_off = [int(t.split("=")[1]) for t in f[2 + 3 ** d:]]
        assert got_off == off
        for p in range(3 ** d):
            v = [(p // 3 ** (d - 1 - a)) % 3 - 1 for a in range(d)]
            delta = sum(v[a] << off[a] for a in range(d)) % 2 ** 64
            vpack = sum((v[a] + 1) << (2 * a) for a in range(d))
            assert f[2 + p] == f"{delta}:{vpack}", (d, spans, p)


def test_plan_from_key_range(planner):
    # the whole plan from a key range (the key-range kernel's input): per axis the key box
    # widened by one cell each side, the fixed-point unit 2^L with
    # L = e + ceil(log2 n) - 126 (max |x| < 2^e), the face-table offsets; and
    # the refusals: |x / h| >= 4e15, more than 2^22 cells on an axis, a packed
    # key wider than 63 bits
    rng = random.Random(9)
    cases = []
    for _ in range(300):
        d = rng.randint(1, 8)
        h = rng.choice(HS)
        n = rng.choice([1, 2, 3, 1000, 1 << 20, (1 << 31) - 1])
        B = rng.choice([1, 1, 5])
        axes = []
        for _ in range(d):
            kind = rng.random()
            if kind < 0.05:
                lo, hi = -5e15 * h, 1.0 * h  # beyond the exact range
            elif kind < 0.1:
                lo, hi = 0.0, h * 5e6  # more than 2^22 cells
            else:
                c = rng.uniform(-1e5, 1e5) * h
                w = rng.choice([0.0, rng.uniform(0, 50), rng.uniform(0, 3000)]) * h
                lo, hi = c, c + w
            axes.append((lo, hi, max(abs(lo), abs(hi))))
        cases.append((d, h, n, B, axes))
    lines = [f"P {d} {h.hex()} {n} {B} " + " ".join(f"{lo.hex()} {hi.hex()} {m.hex()}"
                                                    for lo, hi, m in axes)
             for d, h, n, B, axes in cases]
    out = planner(lines)
    for (d, h, n, B, axes), line in zip(cases, out):
        f = [int(t) for t in line.split()]
        want_status, rows = 0, []
        for lo, hi, m in axes:
            if not (abs(lo / h) < 4.0e15 and abs(hi / h) < 4.0e15):
                want_status = 2
                break
            kmin = math.floor(Fr(lo) / Fr(h)) - 1
            span = math.floor(Fr(hi) / Fr(h)) + 1 - kmin + 1
            if span > 1 << 22:
                want_status = 3
                break
            e = math.frexp(m)[1] if m > 0 else 0
            rows.append((kmin, span, e + (n - 1).bit_length() - 126))
        if want_status == 0:
            bits = sum((s + 1).bit_length() for _, s, _ in rows)
            bits += (B - 1).bit_length() if B > 1 else 0
            if bits > 63:
                want_status = 4
        assert f[0] == want_status, (line, axes)
        if want_status:
            continue
        off = 0
        for a, (kmin, span, L) in enumerate(rows):
            assert f[1 + 4 * a: 5 + 4 * a] == [kmin, span, L, off], (a, axes[a])
            off += span + 1
        assert f[-1] == off
