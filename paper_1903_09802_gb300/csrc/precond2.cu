// The paper's 2-level circulant preconditioner (Section 3.1, eqs. 17-19).
//
// Build: T. Chan's optimal circulant (eq. 13) is applied on the x and y
// levels of each of the six blocks, the z level stays Toeplitz:
//   c2(p, q, r) = sum_{a in {p, p-l}} sum_{b in {q, q-m}} w_l(a) w_m(b) g(a dx, b dx, r dx),
// r = -(n-1) .. n-1, evaluated in FP64 directly at the signed offsets; a 2-D
// DFT over (p, q) block-diagonalises the x and y levels, leaving for every
// frequency pair (wx, wy) one dense 3n x 3n block
//   B[(a, z), (b, z')] = alpha_tilde^{-1} delta - dx^3 Chat2_ab(z - z'; wx, wy),
// which is inverted (Gauss-Jordan with partial pivoting, one CTA per block,
// complex64) and stored: l m (3n)^2 values.  alpha_tilde is that of the first
// right-hand side of the current incidence set.
//
// Apply, restricted to the scatterer like the 3-level form:
// z = M o P2^{-1}(M o v): masked x and y FFTs, per frequency pair the dense
// block times the 3n-vector of (component, z) values, inverse y and x FFTs.
#include <algorithm>
#include <cmath>

#include "fft_kernels.cuh"
#include "plan.hpp"

namespace dda {

namespace {

__device__ const int kA2[6] = {0, 0, 0, 1, 1, 2};
__device__ const int kB2[6] = {0, 1, 2, 1, 2, 2};

// Index of the symmetric block (a, b) in the order xx, xy, xz, yy, yz, zz.
__device__ __forceinline__ int comp_of(int a, int b) {
  if (a > b) {
    const int t = a;
    a = b;
    b = t;
  }
  return a == 0 ? b : (a == 1 ? 2 + b : 5);
}

// c2[comp][rz + n - 1][q][p], FP64.
__global__ void k_chan2(double2* out, long l, long m, long n, double dx, double k) {
  const long nr = 2 * n - 1;
  const long plane = l * m;
  const long tot = plane * nr;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    const long p = i % l, q = (i / l) % m, ri = i / plane;
    const long c = ri - (n - 1);
    double acc[6][2] = {};
    for (int sa = 0; sa < 2; ++sa) {
      if (sa == 1 && p == 0) continue;
      const long a = sa ? p - l : p;
      const double wa = sa ? (double)p / l : (double)(l - p) / l;
      for (int sb = 0; sb < 2; ++sb) {
        if (sb == 1 && q == 0) continue;
        const long b = sb ? q - m : q;
        const double wb = sb ? (double)q / m : (double)(m - q) / m;
        if ((a | b | c) == 0) continue;
        const double w = wa * wb;
        const double X = dx * a, Y = dx * b, Z = dx * c;
        const double r2 = X * X + Y * Y + Z * Z;
        const double rr = sqrt(r2);
        const double rv[3] = {X / rr, Y / rr, Z / rr};
        double sn, cs;
        sincos(k * rr, &sn, &cs);
        const double er = cs / rr, ei = sn / rr;
        for (int cc = 0; cc < 6; ++cc) {
          const double dlt = (kA2[cc] == kB2[cc]) ? 1.0 : 0.0;
          const double pp = rv[kA2[cc]] * rv[kB2[cc]];
          const double qq = (dlt - 3.0 * pp) / r2;
          const double br = k * k * (dlt - pp) - qq;
          const double bi = k * rr * qq;
          acc[cc][0] += w * (er * br - ei * bi);
          acc[cc][1] += w * (er * bi + ei * br);
        }
      }
    }
    for (int cc = 0; cc < 6; ++cc)
      out[(cc * nr + ri) * plane + q * l + p] = make_double2(acc[cc][0], acc[cc][1]);
  }
}

// blocks[f][i][j], f = wy * l + wx, i = a n + z, j = b n + z'.
__global__ void k_assemble2(const double2* __restrict__ chat, float2* __restrict__ blocks, long l,
                            long m, long n, double dx3, double2 at) {
  const long N = 3 * n, plane = l * m, nr = 2 * n - 1;
  const long tot = plane * N * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot;
       t += (long)gridDim.x * blockDim.x) {
    const long f = t / (N * N), ij = t % (N * N);
    const long i = ij / N, j = ij % N;
    const int a = (int)(i / n), b = (int)(j / n);
    const long z = i % n, zp = j % n;
    const double2 c = chat[((long)comp_of(a, b) * nr + (z - zp + n - 1)) * plane + f];
    double2 v = make_double2(-dx3 * c.x, -dx3 * c.y);
    if (i == j) {
      v.x += at.x;
      v.y += at.y;
    }
    blocks[t] = make_float2((float)v.x, (float)v.y);
  }
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place Gauss-Jordan inverse of one N x N complex64 block per CTA, with
// partial (row) pivoting; the row interchanges are undone as column swaps at
// the end.  Pivot row and pivot column are staged in shared memory each step.
__global__ void __launch_bounds__(1024)
    k_gauss_jordan(float2* __restrict__ blocks, int N, int* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rowk = reinterpret_cast<float2*>(smem_raw);  // [N]
  float2* colk = rowk + N;                            // [N]
  int* perm = reinterpret_cast<int*>(colk + N);       // [N]
  __shared__ float s_val[32];
  __shared__ int s_idx[32];
  __shared__ int s_piv;
  float2* A = blocks + (size_t)blockIdx.x * N * N;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5;
  for (int k = 0; k < N; ++k) {
    // pivot: largest |A[i][k]|, i >= k (ties: smallest i)
    float best = -1.f;
    int bi = k;
    for (int i = k + tid; i < N; i += nth) {
      const float2 v = A[(size_t)i * N + k];
      const float a = v.x * v.x + v.y * v.y;
      if (a > best) {
        best = a;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      s_val[wid] = best;
      s_idx[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      float b = -1.f;
      int ii = k;
      for (int w = 0; w < (nth + 31) / 32; ++w)
        if (s_val[w] > b || (s_val[w] == b && s_idx[w] < ii)) {
          b = s_val[w];
          ii = s_idx[w];
        }
      if (!(b > 0.f) || !isfinite(b)) atomicOr(err, 2);
      s_piv = ii;
      perm[k] = ii;
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != k) {
      for (int j = tid; j < N; j += nth) {
        const float2 t = A[(size_t)k * N + j];
        A[(size_t)k * N + j] = A[(size_t)pr * N + j];
        A[(size_t)pr * N + j] = t;
      }
      __syncthreads();
    }
    // pivot row scaled by 1/pivot, with the pivot entry replaced by 1/pivot
    const float2 pv = A[(size_t)k * N + k];
    const float dn = pv.x * pv.x + pv.y * pv.y;
    const float2 inv = make_float2(pv.x / dn, -pv.y / dn);
    for (int j = tid; j < N; j += nth) {
      const float2 v = j == k ? make_float2(1.f, 0.f) : A[(size_t)k * N + j];
      rowk[j] = cmulf(v, inv);
      colk[j] = A[(size_t)j * N + k];
    }
    __syncthreads();
    for (long e = tid; e < (long)N * N; e += nth) {
      const int i = (int)(e / N), j = (int)(e % N);
      if (i == k) {
        A[e] = rowk[j];
      } else {
        const float2 f = colk[i];
        const float2 base = j == k ? make_float2(0.f, 0.f) : A[e];
        const float2 pr2 = cmulf(f, rowk[j]);
        A[e] = make_float2(base.x - pr2.x, base.y - pr2.y);
      }
    }
    __syncthreads();
  }
  // undo the row interchanges as column swaps, last first
  for (int k = N - 1; k >= 0; --k) {
    const int pr = perm[k];
    if (pr != k) {
      for (int i = tid; i < N; i += nth) {
        const float2 t = A[(size_t)i * N + k];
        A[(size_t)i * N + k] = A[(size_t)i * N + pr];
        A[(size_t)i * N + pr] = t;
      }
    }
    __syncthreads();
  }
}

// Per frequency pair f: gather the 3n-vector (component, z) of each right-hand
// side from t[rhs][c][z][f], multiply by the inverse block, scale by 1/(l m)
// (the inverse transforms are unnormalised) and scatter back.
template <typename T>
__global__ void __launch_bounds__(256)
    k_block_apply(cx<T>* __restrict__ t, const float2* __restrict__ blocks, int nrhs, long n,
                  long plane, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long N = 3 * n;
  cx<T>* vin = reinterpret_cast<cx<T>*>(smem_raw);  // [nrhs][N]
  const long f = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (long e = tid; e < (long)nrhs * N; e += blockDim.x) {
    const long r = e / N, i = e % N;
    vin[e] = t[(r * N + i) * plane + f];  // (r, c, z) = r*3n + (c n + z)
  }
  __syncthreads();
  const float2* B = blocks + (size_t)f * N * N;
  for (long i = wid; i < N; i += nw) {
    const float2* row = B + i * N;
    for (int r = 0; r < nrhs; ++r) {
      float ax = 0.f, ay = 0.f;
      for (long j = lane; j < N; j += 32) {
        const float2 b = __ldg(row + j);
        const cx<T> v = vin[(long)r * N + j];
        ax += b.x * (float)v.x - b.y * (float)v.y;
        ay += b.x * (float)v.y + b.y * (float)v.x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o);
        ay += __shfl_down_sync(0xffffffffu, ay, o);
      }
      if (lane == 0) t[((long)r * N + i) * plane + f] = mk<T>(scale * (T)ax, scale * (T)ay);
    }
  }
}

inline unsigned grid_for(long n, int threads) {
  const long g = (n + threads - 1) / threads;
  return (unsigned)std::min<long>(std::max<long>(g, 1), 152L * 32);
}

template <typename T>
void precond2_apply_impl(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s) {
  const cx<T>* tw = tw_of<T>(p);
  cx<T>* t = static_cast<cx<T>*>(p->w.buf2);
  const long l = p->l, m = p->m, n = p->n;
  const long lines = (long)nrhs * 3 * n * m;
  const long plane = l * m;
  launch_contig<T, false>(v, t, p->mat, nullptr, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                          p->Lmax, s);
  if (m > 1)
    launch_strided<T, false>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                             T(1), tw, p->Lmax, s);
  const size_t smem = (size_t)nrhs * 3 * n * sizeof(cx<T>);
  auto kern = k_block_apply<T>;
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  note_launch();
  kern<<<(unsigned)plane, 256, smem, s>>>(t, static_cast<const float2*>(p->w.P2), nrhs, n, plane,
                                          (T)(1.0 / (double)plane));
  if (m > 1)
    launch_strided<T, true>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                            T(1), tw, p->Lmax, s);
  launch_contig<T, true>(t, z, nullptr, p->mat, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                         p->Lmax, s);
}

}  // namespace

template <typename T>
void precond2_apply(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s) {
  precond2_apply_impl<T>(p, nrhs, v, z, s);
}
template void precond2_apply<float>(dda_plan_s*, int, const cx<float>*, cx<float>*, cudaStream_t);
template void precond2_apply<double>(dda_plan_s*, int, const cx<double>*, cx<double>*,
                                     cudaStream_t);

}  // namespace dda

using namespace dda;

extern "C" dda_status_t dda_precond2_build(dda_plan_t p, void* stream) {
  if (!p) return fail(DDA_ERR_INVALID_ARG, "dda_precond2_build: NULL plan");
  if (!p->w.P2) return fail(DDA_ERR_INVALID_ARG, "dda_precond2_build: plan made without precond2");
  if (p->nrhs_inc < 1)
    return fail(DDA_ERR_INVALID_ARG, "dda_precond2_build: set the incidence first (alpha_tilde)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long l = p->l, m = p->m, n = p->n, N = 3 * n;
  double2* c2 = static_cast<double2*>(p->w.C2);
  note_launch();
  k_chan2<<<grid_for(l * m * (2 * n - 1), 128), 128, 0, s>>>(c2, l, m, n, p->d.dx, p->d.k);
  fft3d_inplace<double, false>(reinterpret_cast<cx<double>*>(c2), 6 * (2 * n - 1), (int)l, (int)m, 1,
                               1.0, tw_of<double>(p), p->Lmax, s);
  const double2 at = make_double2(p->ainv_host[0], p->ainv_host[1]);  // rhs 0, entry 0
  const double dx3 = p->d.dx * p->d.dx * p->d.dx;
  note_launch();
  k_assemble2<<<grid_for(l * m * N * N, 256), 256, 0, s>>>(c2, static_cast<float2*>(p->w.P2), l, m,
                                                          n, dx3, at);
  cudaMemsetAsync(p->w.err_flag, 0, 4, s);
  const size_t smem = (size_t)N * (2 * sizeof(float2) + sizeof(int));
  note_launch();
  k_gauss_jordan<<<(unsigned)(l * m), 1024, smem, s>>>(static_cast<float2*>(p->w.P2), (int)N,
                                                      static_cast<int*>(p->w.err_flag));
  int err = 0;
  cudaMemcpyAsync(&err, p->w.err_flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return check_cuda("dda_precond2_build");
  if (err & 2) return fail(DDA_ERR_SINGULAR_PRECOND, "dda_precond2_build: singular block");
  p->precond2_built = true;
  return check_cuda("dda_precond2_build");
}

extern "C" dda_status_t dda_precond2_apply(dda_plan_t p, int32_t prec, int32_t nrhs,
                                           const void* d_v, void* d_z, void* stream) {
  if (!p || !d_v || !d_z) return fail(DDA_ERR_INVALID_ARG, "dda_precond2_apply: NULL argument");
  if (!p->precond2_built)
    return fail(DDA_ERR_NO_PRECOND, "dda_precond2_apply: call dda_precond2_build first");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_precond2_apply: nrhs must be 1..(incidences set)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == DDA_C128 && p->has128) {
    precond2_apply<double>(p, nrhs, static_cast<const cx<double>*>(d_v),
                           static_cast<cx<double>*>(d_z), s);
  } else if (prec == DDA_C64 && p->has64) {
    precond2_apply<float>(p, nrhs, static_cast<const cx<float>*>(d_v), static_cast<cx<float>*>(d_z),
                          s);
  } else {
    return fail(DDA_ERR_INVALID_ARG, "dda_precond2_apply: precision not held by the plan");
  }
  return check_cuda("dda_precond2_apply");
}
