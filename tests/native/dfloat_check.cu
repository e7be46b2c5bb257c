// Host-side check of the library's double-float arithmetic (dfloat.cuh):
// random operands, results compared with the same operations in double on
// the double-float operands' exact values.  Prints the largest relative
// errors of +, -, * and of the double -> double-float round trip.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1903_09802_gb300/csrc/dfloat.cuh"

using dda::df;

int main() {
  std::mt19937_64 rng(12345);
  std::uniform_real_distribution<double> mant(-1.0, 1.0);
  std::uniform_int_distribution<int> ex(-20, 20);
  double e_rt = 0, e_add = 0, e_sub = 0, e_mul = 0;
  for (int t = 0; t < 200000; ++t) {
    const double a = std::ldexp(mant(rng), ex(rng));
    const double b = std::ldexp(mant(rng), ex(rng));
    const df A(a), B(b);
    const double av = (double)A, bv = (double)B;  // exact values of the operands
    if (a != 0) e_rt = std::fmax(e_rt, std::fabs(av - a) / std::fabs(a));
    const double s = av + bv, d = av - bv, p = av * bv;
    if (s != 0) e_add = std::fmax(e_add, std::fabs((double)(A + B) - s) / std::fabs(s));
    if (d != 0) e_sub = std::fmax(e_sub, std::fabs((double)(A - B) - d) / std::fabs(d));
    if (p != 0) e_mul = std::fmax(e_mul, std::fabs((double)(A * B) - p) / std::fabs(p));
  }
  std::printf("%.3e %.3e %.3e %.3e\n", e_rt, e_add, e_sub, e_mul);
  return 0;
}
