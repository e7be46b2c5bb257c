// The 3-level circulant preconditioner P = alpha_tilde^{-1} I - dx^3 C.
//
// Build (Section 3): every one of the six unique BTTB blocks is replaced by
// T. Chan's optimal circulant (eq. 13) on the x, y and z levels in turn,
// which in closed form is
//   c(p,q,r) = sum_{a in {p, p-l}} sum_{b in {q, q-m}} sum_{c in {r, r-n}}
//              w_l(a) w_m(b) w_n(c) g(a dx, b dx, c dx),
//   w_L(p) = (L - p)/L,  w_L(p - L) = p/L   (0 <= p < L),  g(0) = 0,
// evaluated directly at the signed offsets, followed by a 3-D DFT of the
// l x m x n first column (a multilevel circulant is diagonalised by the
// multilevel DFT, Section 3).  The spectrum keeps one octant: C inherits the
// parity of each block on each level.
//
// Apply, restricted to the scatterer (the unknowns of eq. 8 live on
// scatterer voxels; P is the matrix of the box filled with the scatterer's
// material, Section 1): z = M o P^{-1}(M o v) with M the scatterer mask.
// The mask is applied in the first and last passes.  In between: 3-D FFT
// of each field component, the 3x3 symbol
//   Lambda(w) = alpha_tilde^{-1} I - dx^3 Chat(w)
// solved per frequency (closed-form inverse of a complex symmetric 3x3
// matrix), inverse FFT.  Lambda is formed on the fly from the stored Chat and
// the right-hand side's alpha_tilde, so one build serves every incident wave.
#include "precond_apply.cuh"

namespace dda {

namespace {

__device__ const int kA[6] = {0, 0, 0, 1, 1, 2};
__device__ const int kB[6] = {0, 1, 2, 1, 2, 2};

// First column of the 3-level circulant of all six blocks, FP64, layout
// [comp][z][y][x]; T. Chan's (eq. 13) or, with strang, Strang's circulant on
// every level.
__global__ void k_chan3(double2* out, long l, long m, long n, double dx, double k, int strang) {
  pdl_entry();
  const long nvox = l * m * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nvox;
       i += (long)gridDim.x * blockDim.x) {
    const long p = i % l, q = (i / l) % m, r = i / (l * m);
    double acc[6][2] = {};
    for (int sa = 0; sa < 2; ++sa) {
      const double wa = circ_weight(p, l, sa, strang);
      if (wa == 0.0) continue;
      const long a = sa ? p - l : p;
      for (int sb = 0; sb < 2; ++sb) {
        const double wb = circ_weight(q, m, sb, strang);
        if (wb == 0.0) continue;
        const long b = sb ? q - m : q;
        for (int sc = 0; sc < 2; ++sc) {
          const double wc = circ_weight(r, n, sc, strang);
          if (wc == 0.0) continue;
          const long c = sc ? r - n : r;
          if ((a | b | c) == 0) continue;  // g(0) = 0: the self term is alpha^{-1}
          const double w = wa * wb * wc;
          const double X = dx * a, Y = dx * b, Z = dx * c;
          const double r2 = X * X + Y * Y + Z * Z;
          const double rr = sqrt(r2);
          const double rv[3] = {X / rr, Y / rr, Z / rr};
          double sn, cs;
          sincos(k * rr, &sn, &cs);
          const double er = cs / rr, ei = sn / rr;
          for (int cc = 0; cc < 6; ++cc) {
            const double dlt = (kA[cc] == kB[cc]) ? 1.0 : 0.0;
            const double pp = rv[kA[cc]] * rv[kB[cc]];
            const double qq = (dlt - 3.0 * pp) / r2;
            const double br = k * k * (dlt - pp) - qq;
            const double bi = k * rr * qq;
            acc[cc][0] += w * (er * br - ei * bi);
            acc[cc][1] += w * (er * bi + ei * br);
          }
        }
      }
    }
    for (int cc = 0; cc < 6; ++cc) out[cc * nvox + i] = make_double2(acc[cc][0], acc[cc][1]);
  }
}

// Keep 0..l/2, 0..m/2, 0..n/2 of the six spectra, interleaved [..][6].
__global__ void k_compress6(const double2* full, long l, long m, long n, long hx, long hy,
                            long hz, double2* out128, float2* out64) {
  pdl_entry();
  const long H = hx * hy * hz, nvox = l * m * n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < H;
       i += (long)gridDim.x * blockDim.x) {
    const long x = i % hx, y = (i / hx) % hy, z = i / (hx * hy);
    for (int c = 0; c < 6; ++c) {
      const double2 v = full[c * nvox + (z * m + y) * l + x];
      if (out128) out128[i * 6 + c] = v;
      if (out64) out64[i * 6 + c] = make_float2((float)v.x, (float)v.y);
    }
  }
}

inline unsigned grid_for(long n, int threads) {
  const long g = (n + threads - 1) / threads;
  return (unsigned)std::min<long>(std::max<long>(g, 1), 152L * 32);
}

}  // namespace

template void precond_apply_into<float>(dda_plan_s*, int, const cx<float>*, cx<float>*, cx<float>*,
                                        cudaStream_t);
template void precond_apply_impl<float>(dda_plan_s*, int, const cx<float>*, cx<float>*, cudaStream_t);

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_precond_build(dda_plan_t p, void* stream) {
  if (!p) return fail(DDA_ERR_INVALID_ARG, "dda_precond_build: NULL plan");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double2* full = static_cast<double2*>(p->w.buf2);
  note_launch();
  k_chan3<<<grid_for(p->nvox, 128), 128, 0, s>>>(full, p->l, p->m, p->n, p->d.dx, p->d.k,
                                                  p->d.circulant);
  fft3d_inplace<double, false>(reinterpret_cast<cx<double>*>(full), 6, p->l, p->m, p->n, 1.0,
                               tw_of<double>(p), p->Lmax, s);
  note_launch();
  k_compress6<<<grid_for((long)p->cx_ * p->cy_ * p->cz_, 256), 256, 0, s>>>(
      full, p->l, p->m, p->n, p->cx_, p->cy_, p->cz_, static_cast<double2*>(p->w.C128),
      static_cast<float2*>(p->w.C64));
  const dda_status_t st = check_cuda("dda_precond_build");
  if (st == DDA_OK) p->precond_built = true;
  return st;
}

extern "C" dda_status_t dda_precond_apply(dda_plan_t p, int32_t prec, int32_t nrhs, const void* d_v,
                                          void* d_z, void* stream) {
  if (!p || !d_v || !d_z) return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply: NULL argument");
  if (!p->precond_built)
    return fail(DDA_ERR_NO_PRECOND, "dda_precond_apply: call dda_precond_build first");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply: nrhs must be 1..(incidences set)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  ScheduleScope scope(p->sched);
  if (prec == DDA_C128) {
    if (!p->has128) return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply: plan holds no complex128 data");
    precond_apply_impl<double>(p, nrhs, static_cast<const cx<double>*>(d_v),
                               static_cast<cx<double>*>(d_z), s);
  } else if (prec == DDA_C64) {
    if (!p->has64) return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply: plan holds no complex64 data");
    precond_apply_impl<float>(p, nrhs, static_cast<const cx<float>*>(d_v),
                              static_cast<cx<float>*>(d_z), s);
  } else {
    return fail(DDA_ERR_INVALID_ARG, "dda_precond_apply: prec must be DDA_C128 or DDA_C64");
  }
  return check_cuda("dda_precond_apply");
}
