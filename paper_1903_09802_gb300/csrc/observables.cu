// Cross sections of a solution.  The paper prints no formula for them; these
// are the standard DDA expressions of Draine & Flatau for a unit-amplitude
// plane wave, written for the paper's unknowns c (dipole moments p = dx^3 c,
// Draine-Flatau polarizability dx^3 alpha), sums over scatterer voxels:
//   C_ext = 4 pi k dx^3 sum Im(conj(E_inc) . c)
//   C_abs = 4 pi k [ -dx^3 sum Im(alpha^{-1}) |c|^2 - (2/3) k^3 dx^6 sum |c|^2 ]
//   C_sca = 4 pi k [ Im(p^H G p) + (2/3) k^3 dx^6 sum |c|^2 ],
// where p^H G p (G without its diagonal) comes from one complex128 matvec
// y = A c:  dx^3 G c = alpha^{-1} c - y on scatterer voxels, so
//   Im(p^H G p) = dx^3 [ sum Im(alpha^{-1}) |c|^2 - Im sum conj(c) . y ].
// Because G is complex symmetric, Im(p^H G p) = p^H Im(G) p, the quadratic
// form of the scattered power.
#include <algorithm>
#include <cmath>
#include <vector>

#include "plan.hpp"

namespace dda {

namespace {

constexpr int kNT = 256;

__device__ __forceinline__ double warp_sum1(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Per block: S[0] = sum Im(alpha^{-1})|c|^2, S[1] = sum |c|^2,
// S[2] = Im sum conj(c) . y, S[3] = sum Im(conj(E_inc) . c), scatterer only.
__global__ void __launch_bounds__(kNT)
    k_xsec_sums(const double2* __restrict__ c, const double2* __restrict__ y,
                const uint8_t* __restrict__ mat, const double2* __restrict__ ainv, int K1,
                const double* __restrict__ inc, long l, long m, long n, double dx, double k,
                double* __restrict__ part, const double2* __restrict__ pv) {
  pdl_entry();
  __shared__ double sh[4][32];
  const int r = blockIdx.y;
  const long nvox = l * m * n;
  const long chunk = (nvox + gridDim.x - 1) / gridDim.x;
  const long v0 = blockIdx.x * chunk, v1 = min(nvox, v0 + chunk);
  const double* d = inc + r * 6;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (long v = v0 + threadIdx.x; v < v1; v += kNT) {
    const int mt = mat[v];
    if (mt == 0) continue;
    const double2 a = pv != nullptr ? pv[(long)r * nvox + v] : ainv[(long)r * K1 + mt];
    const long x = v % l, yy = (v / l) % m, z = v / (l * m);
    const double px = dx * (x - 0.5 * (l - 1)), py = dx * (yy - 0.5 * (m - 1)),
                 pz = dx * (z - 0.5 * (n - 1));
    double sn, cs;
    sincos(k * (d[0] * px + d[1] * py + d[2] * pz), &sn, &cs);
    for (int q = 0; q < 3; ++q) {
      const double2 cv = c[((long)r * 3 + q) * nvox + v];
      const double2 yv = y[((long)r * 3 + q) * nvox + v];
      const double c2 = cv.x * cv.x + cv.y * cv.y;
      s[0] += a.y * c2;
      s[1] += c2;
      s[2] += cv.x * yv.y - cv.y * yv.x;  // Im(conj(c) y)
      // E_inc_q = pol_q (cos + i sin): Im(conj(E) c) = pol_q (cos c.y - sin c.x)
      s[3] += d[3 + q] * (cs * cv.y - sn * cv.x);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int q = 0; q < 4; ++q) {
    const double t = warp_sum1(s[q]);
    if (lane == 0) sh[q][wid] = t;
  }
  __syncthreads();
  if (wid == 0) {
    for (int q = 0; q < 4; ++q) {
      double t = lane < (kNT >> 5) ? sh[q][lane] : 0.0;
      t = warp_sum1(t);
      if (lane == 0) part[((long)r * gridDim.x + blockIdx.x) * 4 + q] = t;
    }
  }
}

// grad[rhs][0][v] = dC_ext/dRe(eps_v), grad[rhs][1][v] = dC_ext/dIm(eps_v):
// g = (lambda_v . c_v) d(alpha^{-1})/d(eps) (unconjugated over components),
// dRe = pref Im(g), dIm = pref Re(g), pref = -4 pi k dx^3; zero on air.
// With a per-voxel permittivity (eps != null) d(alpha^{-1})/d(eps) is that of
// the voxel's own eps: -4 pi/(eps - 1)^2 + (b2 + b3 S)(k dx)^2, S of the
// right-hand side's wave (inc: direction, polarisation).
__global__ void k_ext_gradient(const double2* __restrict__ c, const double2* __restrict__ lam,
                               const uint8_t* __restrict__ mat, const double2* __restrict__ dainv,
                               int K1, long nvox, int nrhs, double pref, double* __restrict__ grad,
                               const double2* __restrict__ eps, const double* __restrict__ inc,
                               double kd) {
  pdl_entry();
  const long tot = nvox * nrhs;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    const long v = i % nvox, r = i / nvox;
    const int mt = mat[v];
    double gre = 0.0, gim = 0.0;
    if (mt != 0) {
      double sx = 0.0, sy = 0.0;
      for (int q = 0; q < 3; ++q) {
        const double2 a = lam[(r * 3 + q) * nvox + v], b = c[(r * 3 + q) * nvox + v];
        sx += a.x * b.x - a.y * b.y;
        sy += a.x * b.y + a.y * b.x;
      }
      double2 d;
      if (eps != nullptr) {
        const double pi = 3.14159265358979323846;
        const double* q = inc + r * 6;
        double S = 0.0;
        for (int k = 0; k < 3; ++k) S += (q[k] * q[3 + k]) * (q[k] * q[3 + k]);
        const double2 e = eps[v];
        const double ax = e.x - 1.0, ay = e.y;
        const double wx = ax * ax - ay * ay, wy = 2.0 * ax * ay;  // (eps - 1)^2
        const double dn = wx * wx + wy * wy;
        d.x = -4.0 * pi * wx / dn + (0.1648469 + -1.7700004 * S) * kd * kd;
        d.y = 4.0 * pi * wy / dn;
      } else {
        d = dainv[r * K1 + mt];
      }
      const double gx = sx * d.x - sy * d.y, gy = sx * d.y + sy * d.x;
      gre = pref * gy;
      gim = pref * gx;
    }
    grad[(r * 2 + 0) * nvox + v] = gre;
    grad[(r * 2 + 1) * nvox + v] = gim;
  }
}

}  // namespace

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_ext_gradient(dda_plan_t p, int32_t nrhs, const void* d_c,
                                         const void* d_lambda, double* d_grad, void* stream) {
  if (!p || !d_c || !d_lambda || !d_grad)
    return fail(DDA_ERR_INVALID_ARG, "dda_ext_gradient: NULL argument");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_ext_gradient: nrhs must be 1..(incidences set)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double pi = 3.14159265358979323846;
  const double pref = -4.0 * pi * p->d.k * p->d.dx * p->d.dx * p->d.dx;
  const long tot = p->nvox * nrhs;
  const unsigned grid = (unsigned)std::min<long>(std::max<long>((tot + 255) / 256, 1), 152L * 32);
  note_launch();
  k_ext_gradient<<<grid, 256, 0, s>>>(static_cast<const double2*>(d_c),
                                      static_cast<const double2*>(d_lambda), p->mat,
                                      static_cast<const double2*>(p->w.dainv128), p->K + 1,
                                      p->nvox, nrhs, pref, d_grad,
                                      p->voxel_eps_on ? static_cast<const double2*>(p->w.eps_vox)
                                                      : nullptr,
                                      p->w.incd, p->d.k * p->d.dx);
  return check_cuda("dda_ext_gradient");
}

extern "C" dda_status_t dda_cross_sections(dda_plan_t p, int32_t nrhs, const void* d_c,
                                           double* h_out, void* stream) {
  if (!p || !d_c || !h_out) return fail(DDA_ERR_INVALID_ARG, "dda_cross_sections: NULL argument");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_cross_sections: nrhs must be 1..(incidences set)");
  if (!p->has128)
    return fail(DDA_ERR_INVALID_ARG, "dda_cross_sections: plan holds no complex128 data");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cx<double>* c = static_cast<const cx<double>*>(d_c);
  cx<double>* y = static_cast<cx<double>*>(p->w.R128);
  matvec_impl<double>(p, nrhs, c, y, s);
  const int nblk = (int)std::min<long>(304, std::max<long>(1, (p->nvox + 4095) / 4096));
  // partial sums go to the head of buf1 (free once the matvec is done)
  double* part = static_cast<double*>(p->w.buf1);
  note_launch();
  k_xsec_sums<<<dim3(nblk, nrhs), kNT, 0, s>>>(
      reinterpret_cast<const double2*>(c), reinterpret_cast<const double2*>(y), p->mat,
      static_cast<const double2*>(p->w.ainv128), p->K + 1, p->w.incd, p->l, p->m, p->n, p->d.dx,
      p->d.k, part, reinterpret_cast<const double2*>(pv_of<double>(p)));
  std::vector<double> h((size_t)nrhs * nblk * 4);
  cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return check_cuda("dda_cross_sections");
  const double pi = 3.14159265358979323846;
  const double k = p->d.k, dx3 = p->d.dx * p->d.dx * p->d.dx;
  for (int r = 0; r < nrhs; ++r) {
    double S[4] = {0, 0, 0, 0};
    for (int b = 0; b < nblk; ++b)
      for (int q = 0; q < 4; ++q) S[q] += h[((size_t)r * nblk + b) * 4 + q];
    const double rad = (2.0 / 3.0) * k * k * k * dx3 * dx3 * S[1];
    h_out[3 * r + 0] = 4.0 * pi * k * dx3 * S[3];
    h_out[3 * r + 1] = 4.0 * pi * k * (-dx3 * S[0] - rad);
    h_out[3 * r + 2] = 4.0 * pi * k * (dx3 * (S[0] - S[2]) + rad);
  }
  return check_cuda("dda_cross_sections");
}
