"""Accuracy of the double-float (DF64) arithmetic used by the DF64 storage form, on the CPU.

The same header the kernels include is compiled for the host and every operation is compared
with the exactly rounded long-double result on random operands spanning eight decades: the
error stays within a few units of 2^-48 relative to the operands' scale.
"""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = r'''
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <random>
#include "tm_df64.cuh"
using tmk::df64;
static long double ld(df64 a) { return (long double)a.hi + (long double)a.lo; }
int main() {
    std::mt19937_64 rng(12345);
    std::uniform_real_distribution<double> u(-1.0, 1.0), e(-4.0, 4.0);
    double worst[4] = {0, 0, 0, 0}, conv = 0;
    for (int i = 0; i < 200000; i++) {
        double x = u(rng) * std::pow(10.0, e(rng)), y = u(rng) * std::pow(10.0, e(rng)), z = u(rng) * std::pow(10.0, e(rng));
        df64 a(x), b(y), c(z);
        long double la = ld(a), lb = ld(b), lc = ld(c);
        conv = std::fmax(conv, (double)(fabsl(la - x) / fabsl((long double)x)));
        long double scale_ab = fabsl(la) + fabsl(lb), scale_p = fabsl(la * lb);
        worst[0] = std::fmax(worst[0], (double)(fabsl(ld(a + b) - (la + lb)) / scale_ab));
        worst[1] = std::fmax(worst[1], (double)(fabsl(ld(a - b) - (la - lb)) / scale_ab));
        worst[2] = std::fmax(worst[2], (double)(fabsl(ld(a * b) - la * lb) / scale_p));
        worst[3] = std::fmax(worst[3], (double)(fabsl(ld(tmk::fma(a, b, c)) - (la * lb + lc)) / (scale_p + fabsl(lc))));
    }
    printf("%.3e %.3e %.3e %.3e %.3e\n", conv, worst[0], worst[1], worst[2], worst[3]);
    return 0;
}
'''


def test_df64_operations_are_accurate_to_2_pow_minus_48():
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "t.cpp"), os.path.join(d, "t")
        open(src, "w").write(SRC)
        r = subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I",
                            os.path.join(ROOT, "paper_1311_4462_gb300", "csrc"), src, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.fail(r.stderr)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    conv, add, sub, mul, fma = map(float, out)
    u = 2.0 ** -48
    assert conv <= 1.0 * u
    assert add <= 4 * u and sub <= 4 * u
    assert mul <= 4 * u
    assert fma <= 6 * u
