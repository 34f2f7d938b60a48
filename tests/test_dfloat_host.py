"""Float-float arithmetic of the kernels (csrc/dfloat.cuh), checked on the host.

The header's primitives are compiled for the CPU with g++ (IEEE binary32 with
FMA from the C library, no contraction) and compared against long double
references on seeded random inputs: the bounds are those the header states
(sum <= 4u^2 (|x| + |y|) absolute, product <= 12u^2 relative, u = 2^-24; the
FP64 split <= 2^-47 relative with its low part below one ulp of the high part; sin d and 1 - cos d of an angle
increment to absolute errors of 5e-15, the pseudo-Huber ramp to 3e-14
relative to max(1, h)).
No GPU is involved; the kernels use the same source with the _rn intrinsics.
"""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2604_09993_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <random>
#include "dfloat.cuh"
using namespace ciscvx;
typedef long double LD;
static LD v(dflt x) { return (LD)x.h + (LD)x.l; }
int main() {
  std::mt19937_64 g(12345);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> Ex(-20, 20);
  double e_split = 0, e_add = 0, e_mul = 0, e_addf = 0, e_mulf = 0, e_sqr = 0;
  double e_sin_s = 0, e_ver_s = 0, e_sin_l = 0, e_ver_l = 0, e_hub = 0, norm_viol = 0;
  for (int it = 0; it < 200000; ++it) {
    const double a = std::ldexp(U(g), Ex(g)), b = std::ldexp(U(g), Ex(g));
    const dflt x = df_split(a), y = df_split(b);
    if (a != 0.0) e_split = std::fmax(e_split, (double)(std::fabs(v(x) - (LD)a) / std::fabs((LD)a)));
    // the split's low part is below one ulp of the high part
    if (x.h != 0.0f && std::fabs(x.l) >= (std::nextafter(std::fabs(x.h), INFINITY) - std::fabs(x.h)))
      norm_viol += 1;
    const LD s = v(x) + v(y), p = v(x) * v(y);
    e_add = std::fmax(e_add, (double)(std::fabs(v(df_add(x, y)) - s) / (std::fabs(v(x)) + std::fabs(v(y)))));
    if (p != 0) e_mul = std::fmax(e_mul, (double)(std::fabs(v(df_mul(x, y)) - p) / std::fabs(p)));
    if (p != 0) e_sqr = std::fmax(e_sqr, (double)(std::fabs(v(df_sqr(x)) - v(x) * v(x)) / (v(x) * v(x))));
    const float f = (float)b;
    const LD sf = v(x) + (LD)f, pf = v(x) * (LD)f;
    e_addf = std::fmax(e_addf, (double)(std::fabs(v(df_add_f(x, f)) - sf) / (std::fabs(v(x)) + std::fabs((LD)f))));
    if (pf != 0) e_mulf = std::fmax(e_mulf, (double)(std::fabs(v(df_mul_f(x, f)) - pf) / std::fabs(pf)));
    // angle increments
    {
      const dflt d = df_split(0.02 * U(g));
      dflt sn, vc;
      sin_vers_short(d, sn, vc);
      const LD dd = v(d);
      e_sin_s = std::fmax(e_sin_s, (double)std::fabs(v(sn) - std::sin(dd)));
      e_ver_s = std::fmax(e_ver_s, (double)std::fabs(v(vc) - (1.0L - std::cos(dd))));
      const dflt d2 = df_split(0.2 * U(g));
      sin_vers_long(d2, sn, vc);
      const LD d2d = v(d2);
      e_sin_l = std::fmax(e_sin_l, (double)std::fabs(v(sn) - std::sin(d2d)));
      e_ver_l = std::fmax(e_ver_l, (double)std::fabs(v(vc) - (1.0L - std::cos(d2d))));
    }
    {
      const dflt z = df_split(5.5 * U(g) + 4.5);
      const LD zz = v(z), pp = zz > 0 ? zz : 0.0L;
      const LD ref = std::sqrt(1.0L + pp * pp) - 1.0L;
      e_hub = std::fmax(e_hub, (double)(std::fabs(v(huber_df(z)) - ref) / std::fmax(1.0L, ref)));
    }
  }
  std::printf("{\"split\": %.3e, \"add\": %.3e, \"mul\": %.3e, \"sqr\": %.3e, \"add_f\": %.3e, "
              "\"mul_f\": %.3e, \"sin_short\": %.3e, \"vers_short\": %.3e, \"sin_long\": %.3e, "
              "\"vers_long\": %.3e, \"huber\": %.3e, \"norm_violations\": %.0f}\n",
              e_split, e_add, e_mul, e_sqr, e_addf, e_mulf, e_sin_s, e_ver_s, e_sin_l, e_ver_l, e_hub,
              norm_viol);
  return 0;
}
"""


@pytest.fixture(scope="module")
def errors(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("dfloat")
    src, exe = d / "h.cpp", d / "h"
    src.write_text(HARNESS)
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-I", CSRC,
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    return json.loads(out.stdout)


U = 2.0 ** -24


def test_split_of_fp64(errors):
    assert errors["split"] <= 2.0 ** -47
    assert errors["norm_violations"] == 0


def test_sum_and_product_bounds(errors):
    assert errors["add"] <= 4 * U ** 2
    assert errors["add_f"] <= 4 * U ** 2
    assert errors["mul"] <= 12 * U ** 2
    assert errors["mul_f"] <= 12 * U ** 2
    assert errors["sqr"] <= 12 * U ** 2


def test_angle_increment_series(errors):
    assert errors["sin_short"] <= 5e-15 and errors["vers_short"] <= 5e-15
    assert errors["sin_long"] <= 5e-15 and errors["vers_long"] <= 5e-15


def test_pseudo_huber(errors):
    assert errors["huber"] <= 3e-14
