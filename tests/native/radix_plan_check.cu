// Host-side check of the transform plans (fft_core.cuh) and the twiddle
// table length (plan.hpp): prints one line per length L = 2..1024 that is a
// power of two or an even 7-smooth number,
//   "plan <L> <pow2> <hin> <hout> <nst> <r0> ... <r_{nst-1}>",
// and for a few boxes "tw <l> <m> <n> <twiddle_length>".  No GPU work.
#include <cstdio>

#include "../../paper_1903_09802_gb300/csrc/plan.hpp"

using namespace dda;

int main() {
  for (int L = 2; L <= 1024; ++L) {
    if (!is_pow2(L) && !(L % 2 == 0 && is_7smooth(L))) continue;
    const RadixPlan p = make_radix_plan(L);
    std::printf("plan %d %d %d %d %d", L, p.pow2, p.hin, p.hout, p.nst);
    for (int s = 0; s < p.nst; ++s) std::printf(" %d", p.r[s]);
    std::printf("\n");
  }
  const int boxes[][3] = {{64, 64, 128}, {96, 96, 96}, {96, 80, 56}, {6, 10, 14}, {1, 1, 1},
                          {210, 64, 2}};
  for (const auto& b : boxes)
    std::printf("tw %d %d %d %ld\n", b[0], b[1], b[2], twiddle_length(b[0], b[1], b[2]));
  return 0;
}
