"""The double-single arithmetic of the mixed form's residual kernel
(paper_1611_02967_gb300/csrc/chhs_df64.cuh), compiled for the host with the
same source and checked against long double references on random operands
spanning twenty decades: the split of a double into hi + lo, sums and
products must be exact to about 2^-44 relative to the operands, and the
split must keep zero, signs and non-finite values."""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "paper_1611_02967_gb300", "csrc", "chhs_df64.cuh")

PROGRAM = r'''
#include HEADER_PATH
#include <cmath>
#include <cstdio>
#include <random>
using namespace chhs_dev;
int main() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> u(-1, 1);
  long double w_split = 0, w_add = 0, w_mul = 0, w_sub = 0;
  for (int k = 0; k < 300000; ++k) {
    const double x = u(g) * std::pow(10.0, (int)(g() % 20) - 10), y = u(g) * std::pow(10.0, (int)(g() % 20) - 10);
    const df64 a = df_split(x), b = df_split(y);
    const long double ax = (long double)a.hi + a.lo;
    w_split = std::max(w_split, std::fabs(ax - x) / std::fabs((long double)x));
    const df64 s = df_add(a, b), d = df_sub(a, b), p = df_mul(a, b);
    const long double m = std::max(std::fabs((long double)x), std::fabs((long double)y));
    w_add = std::max(w_add, std::fabs((long double)s.hi + s.lo - ((long double)x + y)) / m);
    w_sub = std::max(w_sub, std::fabs((long double)d.hi + d.lo - ((long double)x - y)) / m);
    w_mul = std::max(w_mul, std::fabs((long double)p.hi + p.lo - (long double)x * y) / std::fabs((long double)x * y));
  }
  const df64 z = df_split(0.0), nz = df_split(-0.0), inf = df_split(INFINITY), nan = df_split(NAN);
  const df64 tiny = df_split(1e-40), big = df_split(1e40), neg = df_split(-3.25);
  printf("%Lg %Lg %Lg %Lg %d %d %d %d %d %d %d\n", w_split, w_add, w_sub, w_mul,
         z.hi == 0.f && z.lo == 0.f, std::signbit(nz.hi), std::isinf(inf.hi), std::isinf(nan.hi),
         tiny.hi == 0.f, std::isinf(big.hi), neg.hi == -3.25f && neg.lo == 0.f);
  return 0;
}
'''


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    d = tmp_path_factory.mktemp("df64")
    src = d / "t.cpp"
    src.write_text(PROGRAM.replace("HEADER_PATH", '"%s"' % HEADER))
    exe = d / "t"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    return [float(v) for v in out[:4]] + [int(v) for v in out[4:]]


def test_split_sum_product_accuracy(results):
    w_split, w_add, w_sub, w_mul = results[:4]
    assert w_split <= 2.0 ** -46
    assert w_add <= 2.0 ** -44 and w_sub <= 2.0 ** -44
    assert w_mul <= 2.0 ** -43


def test_split_special_values(results):
    assert results[4:] == [1, 1, 1, 1, 1, 1, 1]
