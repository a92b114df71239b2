"""Double-float primitives of the mixed-precision path (csrc/dd.h), compiled on the host with
contraction disabled, against exact rational arithmetic.

Bounds (u = 2^-24, the FP32 unit roundoff):
* products, quotients, rsqrt: relative error of the result <= 2^-44;
* the exact sum a + b: relative error of the result <= 2^-44 even under cancellation;
* fma_dd (a*b then the exact sum) and fma_dd_fast (one pass, low-order parts summed in FP32):
  error <= 2^-44 (|a b| + |c|), the bound the element terms of the assembly are judged by; the
  fast form must also be correct to that bound under cancellation (a b ~ -c);
* add_acc (the accumulating sum): error <= 2^-44 (|a| + |b|), also under cancellation.
A dropped cross product or low part is an error of order u = 2^-24 and fails every bound."""
import os
import shutil
import subprocess
import textwrap
from fractions import Fraction

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2304_12032_gb300", "csrc")

PROG = textwrap.dedent(r"""
    #include <cstdio>
    #include <cstdlib>
    #include "dd.h"
    using namespace lfx;
    int main() {
      float v[6];
      while (std::scanf("%a %a %a %a %a %a", &v[0], &v[1], &v[2], &v[3], &v[4], &v[5]) == 6) {
        const dd a(v[0], v[1]), b(v[2], v[3]), c(v[4], v[5]);
        const dd r[7] = {a * b, a + b, fma_dd(a, b, c), fma_dd_fast(a, b, c), a / b, dd_rsqrt(dd_abs(a)),
                         add_acc(a, b)};
        for (int k = 0; k < 7; ++k) std::printf("%a %a ", r[k].hi, r[k].lo);
        std::printf("\n");
      }
      return 0;
    }
    """)


@pytest.fixture(scope="module")
def dd_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("dd")
    src = d / "dd_probe.cpp"
    src.write_text(PROG)
    exe = d / "dd_probe"
    subprocess.run([cxx, "-std=c++17", "-O2", "-ffp-contract=off", "-I" + CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


def _rand_dd(rng, n, lo_exp=-8, hi_exp=8):
    hi = (rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(lo_exp, hi_exp, n)) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    ulp = np.spacing(np.abs(hi)).astype(np.float64)
    lo = (rng.uniform(-0.5, 0.5, n) * ulp).astype(np.float32)
    return hi, lo


def _run(exe, rows):
    inp = "\n".join(" ".join(float(x).hex() for x in r) for r in rows) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    res = []
    for line in out:
        if not line.strip():
            continue
        t = [Fraction(float.fromhex(x)) for x in line.split()]
        res.append([t[2 * k] + t[2 * k + 1] for k in range(7)])
    return res


def _exact(h, l):
    return Fraction(float(h)) + Fraction(float(l))


def _check(rows, res):
    bound = Fraction(1, 2 ** 44)
    for r, out in zip(rows, res):
        a, b, c = _exact(r[0], r[1]), _exact(r[2], r[3]), _exact(r[4], r[5])
        prod, s = a * b, a + b
        assert abs(out[0] - prod) <= bound * abs(prod)
        assert abs(out[1] - s) <= bound * abs(s)
        scale = abs(prod) + abs(c)
        assert abs(out[2] - (prod + c)) <= bound * scale
        assert abs(out[3] - (prod + c)) <= bound * scale
        q = a / b
        assert abs(out[4] - q) <= bound * abs(q)
        # rsqrt of |a|: compare squared, y^2 |a| = 1 within 2 x 2^-44
        y = out[5]
        assert abs(y * y * abs(a) - 1) <= 2 * bound
        assert abs(out[6] - s) <= bound * (abs(a) + abs(b))


def test_dd_primitives_random(dd_exe):
    rng = np.random.default_rng(11)
    n = 400
    ah, al = _rand_dd(rng, n)
    bh, bl = _rand_dd(rng, n)
    ch, cl = _rand_dd(rng, n, -4, 12)
    rows = list(zip(ah, al, bh, bl, ch, cl))
    _check(rows, _run(dd_exe, rows))


def test_dd_primitives_cancellation(dd_exe):
    """c close to -a*b (and b close to -a): the sums cancel most of their leading bits."""
    rng = np.random.default_rng(12)
    rows = []
    for _ in range(300):
        ah, al = _rand_dd(rng, 1)
        bh, bl = _rand_dd(rng, 1)
        p = _exact(ah[0], al[0]) * _exact(bh[0], bl[0])
        # -p rounded to a dd, then perturbed in its low part
        neg = -float(p)
        chi = np.float32(neg)
        clo = np.float32(float(Fraction(neg) - Fraction(float(chi))) * (1 + rng.uniform(-1e-3, 1e-3)))
        rows.append((ah[0], al[0], -ah[0], np.float32(al[0] * rng.uniform(-1, 1)), chi, clo))
        rows.append((ah[0], al[0], bh[0], bl[0], chi, clo))
    res = _run(dd_exe, rows)
    bound = Fraction(1, 2 ** 44)
    for r, out in zip(rows, res):
        a, b, c = _exact(r[0], r[1]), _exact(r[2], r[3]), _exact(r[4], r[5])
        s = a + b
        assert abs(out[1] - s) <= bound * abs(s)            # the exact sum keeps relative accuracy
        assert abs(out[6] - s) <= bound * (abs(a) + abs(b))  # the accumulating sum: of the operands
        scale = abs(a * b) + abs(c)
        assert abs(out[2] - (a * b + c)) <= bound * scale
        assert abs(out[3] - (a * b + c)) <= bound * scale
