// The paper's 2-level circulant preconditioner (Section 3, eqs. 17-19; the
// block inversion of Section 3.1).
//
// Build: T. Chan's optimal circulant (eq. 13; Strang's with the plan's
// circulant = 1) is applied on the x and y levels of each of the six blocks,
// the z level stays Toeplitz:
//   c2(p, q, r) = sum_{a in {p, p-l}} sum_{b in {q, q-m}} w_l(a) w_m(b) g(a dx, b dx, r dx),
// r = -(n-1) .. n-1, evaluated in FP64 directly at the signed offsets; a 2-D
// DFT over (p, q) block-diagonalises the x and y levels, leaving for every
// frequency pair (wx, wy) one dense 3n x 3n block
//   B[(a, z), (b, z')] = alpha_tilde^{-1} delta - dx^3 Chat2_ab(z - z'; wx, wy),
// which is inverted (Gauss-Jordan with partial pivoting, one CTA per block,
// complex64; the transpose is assembled and inverted, so the inverse lies in
// memory column-major) and stored.  alpha_tilde is that of the first
// right-hand side of the current incidence set.
//
// Only the quadrant 0 <= wx <= l/2, 0 <= wy <= m/2 is built and stored,
// (l/2 + 1)(m/2 + 1) blocks: every block of the Green tensor is even or odd
// in x and in y (odd in x: xy, xz; odd in y: xy, yz), T. Chan's circulant
// keeps that parity, so its DFT is even or odd in wx and wy, and
//   B(l - wx, wy) = Sx B(wx, wy) Sx,   Sx = diag(-1 on the x component, 1, 1),
// likewise in y; the same holds for the inverse.  The apply flips the signs
// of the x (y) component before and after the product for wx > l/2 (wy > m/2).
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
__global__ void k_chan2(double2* out, long l, long m, long n, double dx, double k, int strang) {
  pdl_entry();
  const long nr = 2 * n - 1;
  const long plane = l * m;
  const long tot = plane * nr;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    const long p = i % l, q = (i / l) % m, ri = i / plane;
    const long c = ri - (n - 1);
    double acc[6][2] = {};
    for (int sa = 0; sa < 2; ++sa) {
      const double wa = circ_weight(p, l, sa, strang);
      if (wa == 0.0) continue;
      const long a = sa ? p - l : p;
      for (int sb = 0; sb < 2; ++sb) {
        const double wb = circ_weight(q, m, sb, strang);
        if (wb == 0.0) continue;
        const long b = sb ? q - m : q;
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

// blocksT[fq][j][i] = B[i][j] (the transpose, whose inverse is the transposed
// inverse the apply reads column-wise), fq = wy * (l/2 + 1) + wx over the
// stored quadrant, i = a n + z, j = b n + z'.
__global__ void k_assemble2(const double2* __restrict__ chat, float2* __restrict__ blocks, long l,
                            long m, long n, double dx3, double2 at) {
  pdl_entry();
  const long N = 3 * n, plane = l * m, nr = 2 * n - 1;
  const long hx = l / 2 + 1, hy = m / 2 + 1;
  const long tot = hx * hy * N * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < tot;
       t += (long)gridDim.x * blockDim.x) {
    const long fq = t / (N * N), ij = t % (N * N);
    const long f = (fq / hx) * l + fq % hx;
    const long j = ij / N, i = ij % N;
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
  pdl_entry();
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
    // a warp per row, lanes along it (coalesced, no index division)
    for (int i = wid; i < N; i += nth >> 5) {
      float2* Ai = A + (size_t)i * N;
      if (i == k) {
        for (int j = lane; j < N; j += 32) Ai[j] = rowk[j];
      } else {
        const float2 f = colk[i];
        for (int j = lane; j < N; j += 32) {
          const float2 base = j == k ? make_float2(0.f, 0.f) : Ai[j];
          const float2 pr2 = cmulf(f, rowk[j]);
          Ai[j] = make_float2(base.x - pr2.x, base.y - pr2.y);
        }
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

// One CTA per stored block (wxq, wyq) serves every frequency pair that mirrors
// onto it (up to four) for right-hand sides r0 .. r0 + nr - 1: it gathers
// those 3n-vectors (component, z) from t[rhs][c][z][wy][wx] into shared
// memory with the mirror's component signs, multiplies them by the block
// (read once, coalesced: blocksT holds each inverse transposed, one thread
// per output row), and scatters the signed, 1/(l m)-scaled results back (the
// inverse transforms are unnormalised).  Vectors are taken VC at a time.
template <typename T, int VC>
__global__ void __launch_bounds__(256)
    k_block_apply(cx<T>* __restrict__ t, const float2* __restrict__ blocksT, int r0, int nr, long l,
                  long m, long n, T scale) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* vin = reinterpret_cast<float2*>(smem_raw);  // [chunk][j][VC]
  const long N = 3 * n, plane = l * m, hx = l / 2 + 1;
  const long fq = blockIdx.x, wxq = fq % hx, wyq = fq / hx;
  const int nfx = (wxq != 0 && 2 * wxq != l) ? 2 : 1;
  const int nfy = (wyq != 0 && 2 * wyq != m) ? 2 : 1;
  const int nf = nfx * nfy, nv = nf * nr, nch = (nv + VC - 1) / VC;
  // vector v: mirror q = v % nf (q % nfx mirrors x, q / nfx mirrors y), rhs v / nf
  for (long e = threadIdx.x; e < (long)nch * N * VC; e += blockDim.x) {
    const int v = (int)(e % VC) + VC * (int)(e / (N * VC));
    const long j = (e / VC) % N;
    float2 x = make_float2(0.f, 0.f);
    if (v < nv) {
      const int q = v % nf, rr = v / nf;
      const bool fx = (q % nfx) != 0, fy = (q / nfx) != 0;
      const long f = (fy ? m - wyq : wyq) * l + (fx ? l - wxq : wxq);
      const long c = j / n;
      const cx<T> a = t[((long)(r0 + rr) * N + j) * plane + f];
      const float sg = ((c == 0 && fx) || (c == 1 && fy)) ? -1.f : 1.f;
      x = make_float2(sg * (float)a.x, sg * (float)a.y);
    }
    vin[e] = x;
  }
  __syncthreads();
  const float2* B = blocksT + (size_t)fq * N * N;
  for (long i = threadIdx.x; i < N; i += blockDim.x) {
    const long c = i / n;
    for (int ch = 0; ch < nch; ++ch) {
      float ax[VC], ay[VC];
#pragma unroll
      for (int s = 0; s < VC; ++s) ax[s] = ay[s] = 0.f;
      const float4* vv = reinterpret_cast<const float4*>(vin + (size_t)ch * N * VC);
#pragma unroll 4
      for (long j = 0; j < N; ++j) {
        const float2 b = __ldg(B + j * N + i);
#pragma unroll
        for (int h = 0; h < VC / 2; ++h) {
          const float4 x = vv[j * (VC / 2) + h];
          ax[2 * h] += b.x * x.x - b.y * x.y;
          ay[2 * h] += b.x * x.y + b.y * x.x;
          ax[2 * h + 1] += b.x * x.z - b.y * x.w;
          ay[2 * h + 1] += b.x * x.w + b.y * x.z;
        }
      }
#pragma unroll
      for (int s = 0; s < VC; ++s) {
        const int v = ch * VC + s;
        if (v < nv) {
          const int q = v % nf, rr = v / nf;
          const bool fx = (q % nfx) != 0, fy = (q / nfx) != 0;
          const long f = (fy ? m - wyq : wyq) * l + (fx ? l - wxq : wxq);
          const T sc = ((c == 0 && fx) || (c == 1 && fy)) ? -scale : scale;
          t[((long)(r0 + rr) * N + i) * plane + f] = mk<T>(sc * (T)ax[s], sc * (T)ay[s]);
        }
      }
    }
  }
}

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  const unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int K>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(K) : "memory");
}

constexpr int kP2Stages = 4;  // tiles in the shared-memory ring
constexpr int kP2Rows = 8;    // block rows per tile

// Multiply-accumulate one block row (b, one value per output row of this
// thread) into the accumulators, against the VC vector entries of that row.
template <int VC, int RPT>
__device__ __forceinline__ void p2_mac(float (&ax)[RPT][VC], float (&ay)[RPT][VC],
                                       const float2 (&b)[RPT], const float4* __restrict__ x4) {
#pragma unroll
  for (int h = 0; h < VC / 2; ++h) {
    const float4 x = x4[h];
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      ax[u][2 * h] = fmaf(b[u].x, x.x, fmaf(-b[u].y, x.y, ax[u][2 * h]));
      ay[u][2 * h] = fmaf(b[u].x, x.y, fmaf(b[u].y, x.x, ay[u][2 * h]));
      ax[u][2 * h + 1] = fmaf(b[u].x, x.z, fmaf(-b[u].y, x.w, ax[u][2 * h + 1]));
      ay[u][2 * h + 1] = fmaf(b[u].x, x.w, fmaf(b[u].y, x.z, ay[u][2 * h + 1]));
    }
  }
}

// The same product with the block streamed through shared memory: tiles of
// kP2Rows block rows are copied with cp.async, kP2Stages - 1 tiles ahead of
// the one being multiplied, so that many bytes are in flight per SM while
// each thread works on RPT output rows from shared memory.  Needs N even
// (16-byte copies) and N <= RPT * blockDim.x.
template <typename T, int VC, int RPT>
__global__ void __launch_bounds__(256)
    k_block_apply_pipe(cx<T>* __restrict__ t, const float2* __restrict__ blocksT, int r0, int nr,
                       long l, long m, long n, T scale) {
  pdl_entry();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 3 * (int)n;
  const long plane = l * m, hx = l / 2 + 1;
  const long fq = blockIdx.x, wxq = fq % hx, wyq = fq / hx;
  const int nfx = (wxq != 0 && 2 * wxq != l) ? 2 : 1;
  const int nfy = (wyq != 0 && 2 * wyq != m) ? 2 : 1;
  const int nf = nfx * nfy, nv = nf * nr, nch = (nv + VC - 1) / VC;
  const int tid = threadIdx.x, nth = blockDim.x;
  float2* sB = reinterpret_cast<float2*>(smem_raw);       // [kP2Stages][kP2Rows][N]
  float2* vin = sB + kP2Stages * kP2Rows * N;            // [chunk][j][VC]
  for (int e = tid; e < nch * N * VC; e += nth) {
    const int v = e % VC + VC * (e / (N * VC));
    const int j = (e / VC) % N;
    float2 x = make_float2(0.f, 0.f);
    if (v < nv) {
      const int q = v % nf, rr = v / nf;
      const bool fx = (q % nfx) != 0, fy = (q / nfx) != 0;
      const long f = (fy ? m - wyq : wyq) * l + (fx ? l - wxq : wxq);
      const int c = j / (int)n;
      const cx<T> a = t[((long)(r0 + rr) * N + j) * plane + f];
      const float sg = ((c == 0 && fx) || (c == 1 && fy)) ? -1.f : 1.f;
      x = make_float2(sg * (float)a.x, sg * (float)a.y);
    }
    vin[e] = x;
  }
  const float2* B = blocksT + (size_t)fq * N * N;
  const int ntiles = (N + kP2Rows - 1) / kP2Rows;
  auto issue = [&](int tile) {
    if (tile < ntiles) {
      const int j0 = tile * kP2Rows;
      const int rows = min(N - j0, kP2Rows);
      const int chunks = rows * N / 2;  // 16-byte pieces
      float2* dst = sB + (tile % kP2Stages) * kP2Rows * N;
      const float2* src = B + (size_t)j0 * N;
      for (int c = tid; c < chunks; c += nth) cp_async16(dst + 2 * c, src + 2 * c);
    }
    cp_async_commit();
  };
  for (int ch = 0; ch < nch; ++ch) {
    float ax[RPT][VC], ay[RPT][VC];
#pragma unroll
    for (int u = 0; u < RPT; ++u)
#pragma unroll
      for (int s = 0; s < VC; ++s) ax[u][s] = ay[u][s] = 0.f;
    const float4* vv = reinterpret_cast<const float4*>(vin + ch * N * VC);
    for (int st = 0; st < kP2Stages - 1; ++st) issue(st);
    for (int tile = 0; tile < ntiles; ++tile) {
      issue(tile + kP2Stages - 1);
      cp_async_wait<kP2Stages - 1>();
      __syncthreads();  // the tile (and, first time round, vin) visible to all threads
      const float2* tb = sB + (tile % kP2Stages) * kP2Rows * N;
      const float4* x4 = vv + tile * kP2Rows * (VC / 2);
      const int rows = min(N - tile * kP2Rows, kP2Rows);
      if (rows == kP2Rows) {
#pragma unroll
        for (int jj = 0; jj < kP2Rows; ++jj) {
          float2 b[RPT];
#pragma unroll
          for (int u = 0; u < RPT; ++u) {
            const int i = tid + u * nth;
            b[u] = (RPT == 1 || i < N) ? tb[jj * N + i] : make_float2(0.f, 0.f);
          }
          p2_mac<VC, RPT>(ax, ay, b, x4 + jj * (VC / 2));
        }
      } else {
        for (int jj = 0; jj < rows; ++jj) {
          float2 b[RPT];
#pragma unroll
          for (int u = 0; u < RPT; ++u) {
            const int i = tid + u * nth;
            b[u] = (RPT == 1 || i < N) ? tb[jj * N + i] : make_float2(0.f, 0.f);
          }
          p2_mac<VC, RPT>(ax, ay, b, x4 + jj * (VC / 2));
        }
      }
      __syncthreads();  // done with this stage before it is refilled
    }
    cp_async_wait<0>();
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const int i = tid + u * nth;
      if (i >= N) continue;
      const int c = i / (int)n;
#pragma unroll
      for (int s = 0; s < VC; ++s) {
        const int v = ch * VC + s;
        if (v < nv) {
          const int q = v % nf, rr = v / nf;
          const bool fx = (q % nfx) != 0, fy = (q / nfx) != 0;
          const long f = (fy ? m - wyq : wyq) * l + (fx ? l - wxq : wxq);
          const T sc = ((c == 0 && fx) || (c == 1 && fy)) ? -scale : scale;
          t[((long)(r0 + rr) * N + i) * plane + f] = mk<T>(sc * (T)ax[u][s], sc * (T)ay[u][s]);
        }
      }
    }
  }
}

// Box the 2-level construction runs on: the plan's own (Toeplitz level z) or
// the relabelled one whose z' is the chosen Toeplitz level, with its mask.
struct P2Geom {
  long l, m, n;
  const uint8_t* mat;
};

// Relabelling of a field batch between the plan's frame and the frame whose
// z' is the Toeplitz level (a rotation: G(R r) = R G(r) R^T):
//   AXIS 2 (x): (x', y', z') = (y, z, x), component c' takes c = {1, 2, 0}[c'];
//   AXIS 3 (y): (x', y', z') = (z, x, y), component c' takes c = {2, 0, 1}[c'].
// TO: dst is in the relabelled frame; otherwise dst is in the plan's frame.
// l, m, n are the plan's edges.
template <typename T, int AXIS, bool TO>
__global__ void k_frame(const cx<T>* __restrict__ src, cx<T>* __restrict__ dst, int nrhs, long l,
                        long m, long n) {
  pdl_entry();
  const long nv = l * m * n, tot = (long)nrhs * 3 * nv;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    const long rc = i / nv, v = i - rc * nv;
    const long r = rc / 3;
    const int c = (int)(rc - 3 * r);
    long sidx;
    int sc;
    if (TO) {
      if (AXIS == 2) {  // frame edges (m, n, l)
        const long xp = v % m, yp = (v / m) % n, zp = v / (m * n);
        sidx = (yp * m + xp) * l + zp;  // (x, y, z) = (z', x', y')
        sc = c == 0 ? 1 : (c == 1 ? 2 : 0);
      } else {  // frame edges (n, l, m)
        const long xp = v % n, yp = (v / n) % l, zp = v / (n * l);
        sidx = (xp * m + zp) * l + yp;  // (x, y, z) = (y', z', x')
        sc = c == 0 ? 2 : (c == 1 ? 0 : 1);
      }
    } else {
      const long x = v % l, y = (v / l) % m, z = v / (l * m);
      if (AXIS == 2) {
        sidx = (x * n + z) * m + y;  // frame (x', y', z') = (y, z, x), edges (m, n, l)
        sc = c == 0 ? 2 : (c == 1 ? 0 : 1);
      } else {
        sidx = (y * l + x) * n + z;  // frame (x', y', z') = (z, x, y), edges (n, l, m)
        sc = c == 0 ? 1 : (c == 1 ? 2 : 0);
      }
    }
    dst[i] = src[(r * 3 + sc) * nv + sidx];
  }
}

// The material mask in the relabelled frame.
template <int AXIS>
__global__ void k_frame_mask(const uint8_t* __restrict__ mat, uint8_t* __restrict__ out, long l,
                             long m, long n) {
  pdl_entry();
  const long nv = l * m * n;
  for (long v = blockIdx.x * (long)blockDim.x + threadIdx.x; v < nv;
       v += (long)gridDim.x * blockDim.x) {
    long sidx;
    if (AXIS == 2) {
      const long xp = v % m, yp = (v / m) % n, zp = v / (m * n);
      sidx = (yp * m + xp) * l + zp;
    } else {
      const long xp = v % n, yp = (v / n) % l, zp = v / (n * l);
      sidx = (xp * m + zp) * l + yp;
    }
    out[v] = mat[sidx];
  }
}

inline P2Geom p2_geom(const dda_plan_s* p) {
  switch (p->d.precond2) {
    case 2: return P2Geom{p->m, p->n, p->l, static_cast<const uint8_t*>(p->w.mat2)};
    case 3: return P2Geom{p->n, p->l, p->m, static_cast<const uint8_t*>(p->w.mat2)};
    default: return P2Geom{p->l, p->m, p->n, p->mat};
  }
}

inline unsigned grid_for(long n, int threads) {
  const long g = (n + threads - 1) / threads;
  return (unsigned)std::min<long>(std::max<long>(g, 1), 152L * 32);
}

template <typename T>
void precond2_apply_impl(dda_plan_s* p, const P2Geom& gm, int nrhs, const cx<T>* v, cx<T>* z,
                         cudaStream_t s) {
  const cx<T>* tw = tw_of<T>(p);
  cx<T>* t = static_cast<cx<T>*>(p->w.buf2);
  const long l = gm.l, m = gm.m, n = gm.n;
  const long lines = (long)nrhs * 3 * n * m;
  const long plane = l * m;
  const double u = (double)nrhs * 3 * p->nvox * sizeof(cx<T>);
  const double blk = (double)(l / 2 + 1) * (m / 2 + 1) * 9.0 * n * n * sizeof(float2);
  // complex128 launches are timed apart from the complex64 ones
  constexpr int pc = std::is_same<T, float>::value ? 0 : PROF_PC128_XF - PROF_PC_XF;
  p->prof.begin(PROF_PC_XF + pc, s, 2 * u + p->nvox);
  launch_contig<T, false>(v, t, gm.mat, nullptr, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                          p->Lmax, s);
  p->prof.end(s);
  p->prof.begin(PROF_PC_YF + pc, s, 2 * u);
  if (m > 1)
    launch_strided<T, false>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                             T(1), tw, p->Lmax, s);
  p->prof.end(s);
  p->prof.begin(PROF_P2_BLOCK, s, 2 * u + blk);
  {
    // right-hand sides per launch: four mirrored vectors each, within shared memory
    const long N = 3 * n;
    const int VC = nrhs == 1 ? 4 : 8;
    const unsigned nq = (unsigned)((l / 2 + 1) * (m / 2 + 1));
    const float2* P2 = static_cast<const float2*>(p->w.P2);
    const T scale = (T)(1.0 / (double)plane);
    const bool pipe = N % 2 == 0 && N <= 512;
    const size_t stage_bytes = pipe ? (size_t)kP2Stages * kP2Rows * N * 8 : 0;
    const auto smem_of = [&](int nr) {
      return stage_bytes + (size_t)((4 * nr + VC - 1) / VC) * VC * N * 8;
    };
    int group = nrhs;
    while (group > 1 && smem_of(group) > 200 * 1024) --group;
    const size_t smem = smem_of(group);
    void (*kern)(cx<T>*, const float2*, int, int, long, long, long, T) = nullptr;
    void (*kpipe)(cx<T>*, const float2*, int, int, long, long, long, T) = nullptr;
    int nth;
    if (pipe) {
      const int rpt = N > 256 ? 2 : 1;
      if (VC == 4)
        kpipe = rpt == 1 ? k_block_apply_pipe<T, 4, 1> : k_block_apply_pipe<T, 4, 2>;
      else
        kpipe = rpt == 1 ? k_block_apply_pipe<T, 8, 1> : k_block_apply_pipe<T, 8, 2>;
      nth = (int)((N / rpt + 31) / 32 * 32);
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(kpipe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    } else {
      kern = VC == 4 ? k_block_apply<T, 4> : k_block_apply<T, 8>;
      nth = (int)std::min<long>(256, (N + 31) / 32 * 32);
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    for (int r0 = 0; r0 < nrhs; r0 += group) {
      const int nr = std::min(group, nrhs - r0);
      note_launch();
      if (pipe)
        launch_k(kpipe, nq, nth, smem, s, t, P2, r0, nr, l, m, n, scale);
      else
        launch_k(kern, nq, nth, smem, s, t, P2, r0, nr, l, m, n, scale);
    }
  }
  p->prof.end(s);
  p->prof.begin(PROF_PC_YI + pc, s, 2 * u);
  if (m > 1)
    launch_strided<T, true>(t, t, l, (long)nrhs * 3 * n, (int)m, (int)m, l, plane, (int)m, l, plane,
                            T(1), tw, p->Lmax, s);
  p->prof.end(s);
  p->prof.begin(PROF_PC_XI + pc, s, 2 * u + p->nvox);
  launch_contig<T, true>(t, z, nullptr, gm.mat, n * m, lines, (int)l, (int)l, l, (int)l, l, T(1), tw,
                         p->Lmax, s);
  p->prof.end(s);
}

}  // namespace

template <typename T>
void precond2_apply_chunk(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s) {
  const P2Geom gm = p2_geom(p);
  const int axis = p->d.precond2;
  if (axis == 1) {
    precond2_apply_impl<T>(p, gm, nrhs, v, z, s);
    return;
  }
  // relabel into buf1 (two box-field batches: in and out), apply, relabel back
  cx<T>* vin = static_cast<cx<T>*>(p->w.buf1);
  cx<T>* vout = vin + (long)nrhs * 3 * p->nvox;
  const unsigned g = grid_for((long)nrhs * 3 * p->nvox, 256);
  note_launch();
  if (axis == 2)
    launch_k(k_frame<T, 2, true>, g, 256, 0, s, v, vin, nrhs, (long)p->l, (long)p->m, (long)p->n);
  else
    launch_k(k_frame<T, 3, true>, g, 256, 0, s, v, vin, nrhs, (long)p->l, (long)p->m, (long)p->n);
  precond2_apply_impl<T>(p, gm, nrhs, vin, vout, s);
  note_launch();
  if (axis == 2)
    launch_k(k_frame<T, 2, false>, g, 256, 0, s, vout, z, nrhs, (long)p->l, (long)p->m, (long)p->n);
  else
    launch_k(k_frame<T, 3, false>, g, 256, 0, s, vout, z, nrhs, (long)p->l, (long)p->m, (long)p->n);
}
// Right-hand sides in chunks of the plan's rhs_chunk (the FFT scratch and
// the relabelling buffers hold that many).
template <typename T>
void precond2_apply(dda_plan_s* p, int nrhs, const cx<T>* v, cx<T>* z, cudaStream_t s) {
  const long nu = 3 * p->nvox;
  for (int r0 = 0; r0 < nrhs; r0 += p->rhs_chunk) {
    const int nr = std::min(p->rhs_chunk, nrhs - r0);
    precond2_apply_chunk<T>(p, nr, v + r0 * nu, z + r0 * nu, s);
  }
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
  if (p->d.precond2 != 1) {
    note_launch();
    if (p->d.precond2 == 2)
      k_frame_mask<2><<<grid_for(p->nvox, 256), 256, 0, s>>>(
          p->mat, static_cast<uint8_t*>(p->w.mat2), p->l, p->m, p->n);
    else
      k_frame_mask<3><<<grid_for(p->nvox, 256), 256, 0, s>>>(
          p->mat, static_cast<uint8_t*>(p->w.mat2), p->l, p->m, p->n);
  }
  const P2Geom gm = p2_geom(p);
  const long l = gm.l, m = gm.m, n = gm.n, N = 3 * n;
  double2* c2 = static_cast<double2*>(p->w.C2);
  note_launch();
  k_chan2<<<grid_for(l * m * (2 * n - 1), 128), 128, 0, s>>>(c2, l, m, n, p->d.dx, p->d.k,
                                                              p->d.circulant);
  fft3d_inplace<double, false>(reinterpret_cast<cx<double>*>(c2), 6 * (2 * n - 1), (int)l, (int)m, 1,
                               1.0, tw_of<double>(p), p->Lmax, s);
  const double2 at = make_double2(p->ainv_host[0], p->ainv_host[1]);  // rhs 0, entry 0
  const double dx3 = p->d.dx * p->d.dx * p->d.dx;
  const long nq = (l / 2 + 1) * (m / 2 + 1);  // stored quadrant of frequency pairs
  note_launch();
  k_assemble2<<<grid_for(nq * N * N, 256), 256, 0, s>>>(c2, static_cast<float2*>(p->w.P2), l, m, n,
                                                       dx3, at);
  cudaMemsetAsync(p->w.err_flag, 0, 4, s);
  const size_t smem = (size_t)N * (2 * sizeof(float2) + sizeof(int));
  note_launch();
  k_gauss_jordan<<<(unsigned)nq, 1024, smem, s>>>(static_cast<float2*>(p->w.P2), (int)N,
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
  ScheduleScope scope(p->sched);
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
