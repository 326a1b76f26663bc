"""The double-float arithmetic of the exact emission solve (csrc/dfloat.cuh),
compiled for the host with g++ (binary32 arithmetic without contraction,
the same operations the device performs), against the host's extended
precision: the error-free transformations are exact, expm1 and its
reciprocal keep ~1e-14 relative over the range the solve uses
(x = a_l / T from 7e-3 to 70), and e - 1 comes out right."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1705_04702_gb300", "csrc", "dfloat.cuh")

HARNESS = r"""
#include <stdio.h>
#include <stdlib.h>
#include <math.h>
#include "dfloat.cuh"
using namespace dfl;
static df2 split(double x) { float h = (float)x; return make(h, (float)(x - (double)h)); }
static long double val(df2 v) { return (long double)v.hi + (long double)v.lo; }
int main(int argc, char** argv) {
    int n = atoi(argv[1]);
    srand(7);
    double w_e = 0, w_q = 0, w_sum = 0, w_prod = 0;
    for (int k = 0; k < n; ++k) {
        double u = (double)rand() / RAND_MAX;
        double x = (k % 2) ? 7e-3 * pow(70.0 / 7e-3, u) : 70.0 * u;
        df2 xd = split(x);
        long double xx = val(xd), ref = expm1l(xx);
        df2 e = expm1(xd);
        double re = (double)(fabsl(val(e) - ref) / ref);
        if (re > w_e) w_e = re;
        df2 q = recip(e);
        double rq = (double)(fabsl(val(q) - 1.0L / ref) * ref);
        if (rq > w_q) w_q = rq;
        float a = (float)(u * 3.0 - 1.5), b = (float)((double)rand() / RAND_MAX * 2.0 - 1.0);
        float s, t;
        two_sum(a, b, s, t);
        double ds = (double)fabsl(((long double)s + t) - ((long double)a + b));
        if (ds > w_sum) w_sum = ds;
        two_prod(a, b, s, t);
        double dp = (double)fabsl(((long double)s + t) - (long double)a * b);
        if (dp > w_prod) w_prod = dp;
    }
    df2 e1 = expm1(make(1.0f, 0.0f));
    printf("%.17g %.17g %.17g %.17g %.21Lg\n", w_e, w_q, w_sum, w_prod, val(e1));
    return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("dfloat")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True)
    return exe


def test_double_float_expm1_and_reciprocal(harness):
    out = subprocess.run([str(harness), "400000"], check=True, capture_output=True, text=True).stdout.split()
    w_e, w_q, w_sum, w_prod = (float(v) for v in out[:4])
    assert w_sum == 0.0 and w_prod == 0.0  # error-free transformations
    assert w_e < 4e-14, w_e
    assert w_q < 4e-14, w_q
    # e - 1 = 1.718281828459045235360287... (the argument 1 is exact in binary32)
    assert abs(float(out[4]) - 1.718281828459045235360287) < 4e-14
