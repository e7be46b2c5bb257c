// s-step GMRES (method 2): the kernels of one block of s columns and the
// shifts.  Included by krylov.cu inside its anonymous namespace (it uses the
// accumulators, pair loads, chunking, Givens rotation and loop control
// defined there).
//
// One block of a cycle starts at column j with q_j (in the fixed buffer Z):
//   for t < s:  W_t = A P^{-1} W_{t-1} - theta_t W_{t-1}  (W_{-1} = q_j;
//               preconditioner, matvec, k_shift)         [Bai, Hu & Reichel 1994]
//   pass 1:     C1 = Q_j^H W, W -= Q_j C1                (k_sdots, k_sdots_reduce, k_supd)
//   pass 2:     C2 = Q_j^H W and G = W^H W               (k_sdots with the Gram rows)
//   k_ssmall:   R from G - C2^H C2 = R^H R (Cholesky), the block's Hessenberg
//               columns (Rc B - [H_j Rc_top; 0]) Rc_bot^{-1} (Hoemmen 2010,
//               Sec. 3.3), then the Givens rotations and the convergence test
//               of each new column
//   final:      q_{j+1..j+s} = (W - Q_j C2) R^{-1} into the basis and q_{j+s}
//               into Z (k_supd)
// Dots read the basis once per pass for all s vectors: four basis passes per
// s columns, against two or more per column for Arnoldi.

constexpr int kBNT = 256;     // threads of the block dot-product kernel
constexpr int kSMax = 8;      // largest block
constexpr int kSRestart = 64; // largest restart of method 2 (shared-memory tables)

// Exact products into a compensated FP32 sum (the Gram matrix of the block
// must be accurate well below FP32 rounding for its Cholesky factor).
struct ExactAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = x * y;
    const float e = fmaf(x, y, -p);
    float t, e2;
    two_sum(s, p, t, e2);
    s = t;
    c += e + e2;
  }
  __device__ __forceinline__ double warp_total() const { return warp_sum_comp(s, c); }
};

// Basis rows: the dot products of NV basis vectors q_{i0..i0+NV-1} (those
// <= j) with the block's S vectors over [k0, k1), out[i * S + t] (lane 0
// writes).  Each W pair loaded (through L1: the block's warps share the
// chunk) serves NV basis vectors.  Plain sums per lane in the working
// precision: only pass 2's coefficients enter the result with their
// rounding (pass 1's are corrected by pass 2), and those are tiny.
template <typename T, int S, int NV>
__device__ __forceinline__ void sdots_basis(const cx<T>* __restrict__ vb, int i0, int j,
                                            long vstride, const cx<T>* __restrict__ wr, long k0,
                                            long k1, int lane, double2* __restrict__ out) {
  T re[NV][S], im[NV][S];
#pragma unroll
  for (int v = 0; v < NV; ++v)
#pragma unroll
    for (int t = 0; t < S; ++t) re[v][t] = im[v][t] = (T)0;
  // two trips per iteration, all their basis loads issued before the first
  // use (the second trip masked at the end of the chunk)
  for (long k = k0 + 2 * lane; k < k1; k += 128) {
    const bool two = k + 64 < k1;
    Pair<T> q[2][NV];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v)
        q[u][v] = (i0 + v <= j && (u == 0 || two))
                      ? ld2_na(vb + (long)(i0 + v) * vstride + k + 64 * u)
                      : Pair<T>{zero<T>(), zero<T>()};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
#pragma unroll
      for (int t = 0; t < S; ++t) {
        const Pair<T> w = ld2(wr + t * vstride + k + 64 * u);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const Pair<T>& a = q[u][v];
          re[v][t] += a.a.x * w.a.x + a.a.y * w.a.y + a.b.x * w.b.x + a.b.y * w.b.y;
          im[v][t] += a.a.x * w.a.y - a.a.y * w.a.x + a.b.x * w.b.y - a.b.y * w.b.x;
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
#pragma unroll
    for (int t = 0; t < S; ++t) {
      T x = re[v][t], y = im[v][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
      }
      if (lane == 0 && i0 + v <= j) out[(i0 + v) * S + t] = make_double2((double)x, (double)y);
    }
  }
}

// Gram row a: <W_a, W_t> for t >= a (zeros for t < a; the matrix is
// Hermitian), out[t].  In complex64 the products are exact (FMA residual)
// and summed with compensation: the Cholesky factor of the block needs the
// Gram matrix far below FP32 rounding.
template <typename T, int S>
__device__ __forceinline__ void sdots_gram(const cx<T>* __restrict__ wr, int a, long vstride,
                                           long k0, long k1, int lane, double2* __restrict__ out) {
  const cx<T>* wa = wr + (long)a * vstride;
  if constexpr (sizeof(T) == 8) {
    double re[S], im[S];
#pragma unroll
    for (int t = 0; t < S; ++t) re[t] = im[t] = 0.0;
    for (long k = k0 + 2 * lane; k < k1; k += 64) {
      const Pair<T> p = ld2(wa + k);
#pragma unroll
      for (int t = 0; t < S; ++t) {
        if (t < a) continue;
        const Pair<T> w = ld2(wr + t * vstride + k);
        re[t] += p.a.x * w.a.x + p.a.y * w.a.y + p.b.x * w.b.x + p.b.y * w.b.y;
        im[t] += p.a.x * w.a.y - p.a.y * w.a.x + p.b.x * w.b.y - p.b.y * w.b.x;
      }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const double2 v = warp_sum(make_double2(re[t], im[t]));
      if (lane == 0) out[t] = t < a ? make_double2(0.0, 0.0) : v;
    }
  } else {
    ExactAcc re[S], im[S];
    for (long k = k0 + 2 * lane; k < k1; k += 64) {
      const Pair<T> p = ld2(wa + k);
#pragma unroll
      for (int t = 0; t < S; ++t) {
        if (t < a) continue;
        const Pair<T> w = ld2(wr + t * vstride + k);
        re[t].add_prod(p.a.x, w.a.x);
        re[t].add_prod(p.a.y, w.a.y);
        re[t].add_prod(p.b.x, w.b.x);
        re[t].add_prod(p.b.y, w.b.y);
        im[t].add_prod(p.a.x, w.a.y);
        im[t].add_prod(-p.a.y, w.a.x);
        im[t].add_prod(p.b.x, w.b.y);
        im[t].add_prod(-p.b.y, w.b.x);
      }
    }
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const double vr = re[t].warp_total(), vi = im[t].warp_total();
      if (lane == 0) out[t] = t < a ? make_double2(0.0, 0.0) : make_double2(vr, vi);
    }
  }
}

// Block partial sums: part[(r * nb + blk) * slots + i * S + t] for the
// basis vectors i <= j (tasks of NV vectors) and, with gram, the rows
// i = j + 1 + a of the block's Gram matrix (one task each); one warp per
// task.  Needs an even vector length (16-byte pairs).
template <typename T, int S>
__global__ void __launch_bounds__(kBNT, sizeof(T) == 4 ? 3 : 1)
    k_sdots(const cx<T>* __restrict__ V, const cx<T>* __restrict__ Wb, long nu, long vstride,
            int j, const int* __restrict__ jdev, int gram, const int* __restrict__ mask,
            double2* __restrict__ part, int slots) {
  pdl_entry();
  if (jdev != nullptr) j = *jdev;
  const int r = blockIdx.y;
  if (!mask[r]) return;
  constexpr int NW = kBNT / 32;
  constexpr int NV = S <= 3 ? 3 : 2;  // basis vectors per task
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  const cx<T>* wr = Wb + r * nu;
  const int nbt = (j + NV) / NV;
  const int ntask = nbt + (gram ? S : 0);
  double2* out = part + ((long)r * gridDim.x + blockIdx.x) * slots;
  // Gram tasks first: they are the longest in complex64
  for (int task = wid; task < ntask; task += NW) {
    if (gram && task < S)
      sdots_gram<T, S>(wr, task, vstride, k0, k1, lane, out + (j + 1 + task) * S);
    else
      sdots_basis<T, S, NV>(V + r * nu, (task - (gram ? S : 0)) * NV, j, vstride, wr, k0, k1,
                            lane, out);
  }
}

// Sum of the blocks' partials in a fixed order: one warp per slot, lanes over
// the blocks; cb[(r * 2 + pass) * cst + slot].
__global__ void __launch_bounds__(256)
    k_sdots_reduce(const double2* __restrict__ part, int nb, int slots, int S, int j,
                   const int* __restrict__ jdev, int gram, const int* __restrict__ mask,
                   double2* __restrict__ cb, int cst, int pass) {
  pdl_entry();
  if (jdev != nullptr) j = *jdev;
  const int r = blockIdx.y;
  if (!mask[r]) return;
  const int lane = threadIdx.x & 31;
  const int slot = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (slot >= (j + 1 + (gram ? S : 0)) * S) return;
  double2 a = make_double2(0.0, 0.0);
  for (int b = lane; b < nb; b += 32) {
    const double2 v = part[((long)r * nb + b) * slots + slot];
    a.x += v.x;
    a.y += v.y;
  }
  a = warp_sum(a);
  if (lane == 0) cb[((long)r * 2 + pass) * cst + slot] = a;
}

// W_t -= sum_{i <= j} C[i][t] q_i for t < S (pass 1, C from cb pass 0, W
// rewritten), or the block's final vectors: x = (W - Q_j C2) R^{-1} into the
// basis slots j+1 .. j+S (and x_{S-1} into Zc).  With jdev the block start is
// *jdev - jshift (the small kernel has advanced the step index by S).
// Thread per 16-byte pair; basis pairs loaded four at a time.
template <typename T, int S>
__global__ void __launch_bounds__(kNT)
    k_supd(cx<T>* __restrict__ V, cx<T>* __restrict__ Wb, long nu, long vstride, int j,
           const int* __restrict__ jdev, int jshift, const double2* __restrict__ cb, int cst,
           int pass, const double2* __restrict__ rinv, const int* __restrict__ mask,
           cx<T>* __restrict__ Zc) {
  pdl_entry();
  if (jdev != nullptr) j = *jdev - jshift;
  const int r = gridDim.y - 1 - blockIdx.y;
  if (!mask[r]) return;
  __shared__ cx<T> cs[(kSRestart + 1) * S];
  __shared__ cx<T> ri[S * S];
  const double2* c = cb + ((long)r * 2 + pass) * cst;
  for (int i = threadIdx.x; i < (j + 1) * S; i += kNT) cs[i] = mk<T>((T)c[i].x, (T)c[i].y);
  const bool fin = rinv != nullptr;
  if (fin)
    for (int i = threadIdx.x; i < S * S; i += kNT) {
      const double2 v = rinv[(long)r * 64 + i];
      ri[i] = mk<T>((T)v.x, (T)v.y);
    }
  __syncthreads();
  long k0, k1;
  {
    // backwards over the chunks: the dots pass just walked the basis forwards
    long chunk = (nu + gridDim.x - 1) / gridDim.x;
    chunk += chunk & 1;
    k0 = min(nu, (long)(gridDim.x - 1 - blockIdx.x) * chunk);
    k1 = min(nu, k0 + chunk);
  }
  cx<T>* wr = Wb + r * nu;
  const cx<T>* vb = V + r * nu;
  for (long k = k0 + 2 * threadIdx.x; k < k1; k += 2 * kNT) {
    Pair<T> w[S];
#pragma unroll
    for (int t = 0; t < S; ++t) w[t] = ld2(wr + t * vstride + k);
    for (int i = 0; i <= j; i += 4) {
      Pair<T> q[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i + u <= j) q[u] = ld2_na(vb + (long)(i + u) * vstride + k);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (i + u <= j) {
#pragma unroll
          for (int t = 0; t < S; ++t) {
            const cx<T> h = cs[(i + u) * S + t];
            w[t].a = w[t].a - h * q[u].a;
            w[t].b = w[t].b - h * q[u].b;
          }
        }
      }
    }
    if (fin) {
      cx<T>* vo = V + r * nu + (long)(j + 1) * vstride + k;
#pragma unroll
      for (int t = 0; t < S; ++t) {
        Pair<T> x{zero<T>(), zero<T>()};
#pragma unroll
        for (int u = 0; u <= t; ++u) {
          const cx<T> f = ri[u * S + t];
          x.a = x.a + f * w[u].a;
          x.b = x.b + f * w[u].b;
        }
        st2(vo + (long)t * vstride, x);
        if (t == S - 1 && Zc != nullptr) st2(Zc + r * nu + k, x);
      }
    } else {
#pragma unroll
      for (int t = 0; t < S; ++t) st2(wr + t * vstride + k, w[t]);
    }
  }
}

// The Newton step's shift: W_t -= theta_t x (x the step's input).
template <typename T>
__global__ void __launch_bounds__(kNT)
    k_shift(cx<T>* __restrict__ Wt, const cx<T>* __restrict__ x, long nu,
            const double2* __restrict__ theta, int t, const int* __restrict__ active) {
  pdl_entry();
  const int r = blockIdx.y;
  if (!active[r]) return;
  const double2 th = theta[(long)r * kSMax + t];
  const cx<T> f = mk<T>((T)th.x, (T)th.y);
  long k0, k1;
  chunk_of(nu, gridDim.x, k0, k1);
  for (long k = k0 + threadIdx.x; k < k1; k += kNT) Wt[r * nu + k] = Wt[r * nu + k] - f * x[r * nu + k];
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 conj2(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}

// After pass 2, one warp per right-hand side (FP64): the Cholesky factor R of
// the block's Gram matrix (with G - C2^H C2 = R^H R: the Gram matrix of
// W - Q C2 when Q is orthonormal), its inverse (for k_supd), the Hessenberg
// columns j .. j+S-1 (unrotated into Hraw, rotated into H), and per column the
// Givens rotation, residual estimate and the tests of k_givens.  A Gram
// matrix that is not numerically positive definite ends the cycle before the
// block (breakdown flag).  blkmask[r] = 1 for the right-hand sides that ran
// the block (their final vectors are written).  The last block advances the
// step index by S and sets the condition of the next block.  Dynamic shared
// memory: (j+S+1) S (Hn) + (j+1) S (C) + 3 S^2 double2 plus the rotations.
__global__ void __launch_bounds__(32)
    k_ssmall(int S, double2* __restrict__ Hraw, double2* __restrict__ H,
             double* __restrict__ cs, double2* __restrict__ sn, double2* __restrict__ g,
             double* __restrict__ scal, int* __restrict__ active, int* __restrict__ blkmask,
             int* __restrict__ jlen, int* __restrict__ flags, int* __restrict__ iters,
             const double2* __restrict__ cb, int cst, double2* __restrict__ rinv,
             const double2* __restrict__ theta, int nrhs, int m, int j, double brk,
             int* __restrict__ count_out, int* __restrict__ ticket, LoopCtl ctl) {
  pdl_entry();
  if (ctl.graph) j = *ctl.jstep;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nrow = j + S + 1;
  double2* Hn = reinterpret_cast<double2*>(smem_raw);  // [nrow][S]
  double2* Cm = Hn + nrow * S;                          // [j+1][S]
  double2* Gm = Cm + (j + 1) * S;                       // [S][S]
  double2* Rm = Gm + S * S;                             // [S][S]
  double2* Ri = Rm + S * S;                             // [S][S]
  double2* hs = Ri + S * S;                             // [nrow] one column
  double2* ss = hs + nrow;                              // [j+S] rotations
  double* cc = reinterpret_cast<double*>(ss + (j + S));
  __shared__ int s_ok;
  const int r = blockIdx.x, lane = threadIdx.x;
  if (active[r]) {
    if (lane == 0) blkmask[r] = 1;
    const double2* c1 = cb + (long)r * 2 * cst;
    const double2* c2 = c1 + cst;
    for (int i = lane; i < (j + 1) * S; i += 32) Cm[i] = cadd(c1[i], c2[i]);
    for (int e = lane; e < S * S; e += 32) {
      const int a = e / S, b = e - a * S;
      // <W_a, W_b>: the dots hold the upper triangle
      double2 v = b >= a ? c2[(j + 1 + a) * S + b] : conj2(c2[(j + 1 + b) * S + a]);
      for (int i = 0; i <= j; ++i) v = csub(v, cmulc(c2[i * S + a], c2[i * S + b]));
      Gm[e] = v;
    }
    __syncwarp();
    if (lane == 0) {
      // Cholesky of D^-1 G D^-1 (D the diagonal's square roots), R = U D
      int ok = 1;
      double d[kSMax];
      for (int a = 0; a < S; ++a) {
        const double ga = Gm[a * S + a].x;
        d[a] = ga > 0.0 ? sqrt(ga) : 0.0;
        if (!(d[a] > 0.0) || !isfinite(d[a])) ok = 0;
      }
      for (int a = 0; a < S && ok; ++a) {
        double diag = Gm[a * S + a].x / (d[a] * d[a]);
        for (int u = 0; u < a; ++u) diag -= Rm[u * S + a].x * Rm[u * S + a].x + Rm[u * S + a].y * Rm[u * S + a].y;
        if (!(diag > 1e-24)) {
          ok = 0;
          break;
        }
        const double ua = sqrt(diag);
        Rm[a * S + a] = make_double2(ua, 0.0);
        for (int b = a + 1; b < S; ++b) {
          double2 v = Gm[a * S + b];
          v = make_double2(v.x / (d[a] * d[b]), v.y / (d[a] * d[b]));
          for (int u = 0; u < a; ++u) v = csub(v, cmulc(Rm[u * S + a], Rm[u * S + b]));
          Rm[a * S + b] = make_double2(v.x / ua, v.y / ua);
        }
        for (int b = 0; b < a; ++b) Rm[a * S + b] = make_double2(0.0, 0.0);
      }
      if (ok) {
        for (int a = 0; a < S; ++a)
          for (int b = a; b < S; ++b) Rm[a * S + b] = make_double2(Rm[a * S + b].x * d[b], Rm[a * S + b].y * d[b]);
        // R^{-1} (upper triangular), column by column
        for (int b = 0; b < S; ++b) {
          for (int a = S - 1; a >= 0; --a) {
            double2 v = make_double2(a == b ? 1.0 : 0.0, 0.0);
            for (int u = a + 1; u <= b; ++u) v = csub(v, cmul(Rm[a * S + u], Ri[u * S + b]));
            Ri[a * S + b] = a > b ? make_double2(0.0, 0.0) : cdiv(v, Rm[a * S + a]);
          }
        }
        for (int e = 0; e < S * S; ++e) rinv[(long)r * 64 + e] = Ri[e];
      }
      s_ok = ok;
    }
    __syncwarp();
    if (!s_ok) {
      if (lane == 0) {
        flags[r] |= 2;  // the block is numerically dependent: the cycle ends before it
        active[r] = 0;
        blkmask[r] = 0;
      }
    } else {
      const double2* th = theta + (long)r * kSMax;
      const double2* hr = Hraw + (long)r * (m + 1) * m;
      // Rc(row, u): [v_0 .. v_S] = [Q_j, Q_new] Rc
      auto rc = [&](int row, int u) -> double2 {
        if (u == 0) return make_double2(row == j ? 1.0 : 0.0, 0.0);
        if (row <= j) return Cm[row * S + u - 1];
        const int a = row - j - 1;
        return a <= u - 1 ? Rm[a * S + u - 1] : make_double2(0.0, 0.0);
      };
      for (int row = lane; row < nrow; row += 32) {
        double2 mrow[kSMax];
        for (int t = 0; t < S; ++t) {
          double2 v = cadd(cmul(th[t], rc(row, t)), rc(row, t + 1));
          if (row <= j && t >= 1) {
            // - (H_j Rc_top)[row][t]: H_j's row `row` is non-zero in columns >= row - 1
            for (int c = max(0, row - 1); c < j; ++c)
              v = csub(v, cmul(hr[(long)c * (m + 1) + row], Cm[c * S + t - 1]));
          }
          mrow[t] = v;
        }
        // X Rc_bot = M, Rc_bot[u][t] = Rc(j + u, t)
        for (int t = 0; t < S; ++t) {
          double2 v = mrow[t];
          for (int u = 0; u < t; ++u) v = csub(v, cmul(Hn[row * S + u], rc(j + u, t)));
          const double2 x = cdiv(v, rc(j + t, t));
          Hn[row * S + t] = row > j + t + 1 ? make_double2(0.0, 0.0) : x;
        }
      }
      __syncwarp();
      for (int e = lane; e < nrow * S; e += 32) {
        const int row = e / S, t = e - row * S;
        if (row <= j + t + 1) Hraw[(long)r * (m + 1) * m + (long)(j + t) * (m + 1) + row] = Hn[e];
      }
      // rotations of the earlier columns
      for (int i = lane; i < j; i += 32) {
        ss[i] = sn[(long)r * m + i];
        cc[i] = cs[(long)r * m + i];
      }
      __syncwarp();
      if (lane == 0) {
        double* sc = scal + (long)r * 16;
        double2* gg = g + (long)r * (m + 1);
        for (int t = 0; t < S; ++t) {
          const int col = j + t;
          for (int i = 0; i <= col + 1; ++i) hs[i] = Hn[i * S + t];
          double colnorm2 = 0.0;
          for (int i = 0; i <= col + 1; ++i) colnorm2 += hs[i].x * hs[i].x + hs[i].y * hs[i].y;
          for (int i = 0; i < col; ++i) {
            const double2 a = hs[i], b = hs[i + 1], si = ss[i];
            const double ci = cc[i];
            hs[i] = make_double2(ci * a.x + (si.x * b.x - si.y * b.y),
                                 ci * a.y + (si.x * b.y + si.y * b.x));
            hs[i + 1] = make_double2(-(si.x * a.x + si.y * a.y) + ci * b.x,
                                     -(si.x * a.y - si.y * a.x) + ci * b.y);
          }
          const double hn = hypot(hs[col + 1].x, hs[col + 1].y);
          double cj;
          double2 sj, rho;
          givens(hs[col], hs[col + 1], cj, sj, rho);
          cc[col] = cj;
          ss[col] = sj;
          cs[(long)r * m + col] = cj;
          sn[(long)r * m + col] = sj;
          hs[col] = rho;
          hs[col + 1] = make_double2(0.0, 0.0);
          double2* h = H + (long)r * (m + 1) * m + (long)col * (m + 1);
          for (int i = 0; i <= col + 1; ++i) h[i] = hs[i];
          const double2 gj = gg[col];
          gg[col + 1] = make_double2(-(sj.x * gj.x + sj.y * gj.y), -(sj.x * gj.y - sj.y * gj.x));
          gg[col] = make_double2(cj * gj.x, cj * gj.y);
          const double res = hypot(gg[col + 1].x, gg[col + 1].y);
          sc[4] = res;
          jlen[r] = col + 1;
          const int it = iters[r] + 1;
          iters[r] = it;
          if (ctl.hist != nullptr && it < ctl.hcap) {
            const double bn = sc[2];
            ctl.hist[(long)r * ctl.hcap + it] = bn > 0.0 ? res / bn : res;
          }
          bool stop = true;
          if (ctl.timeout_ns > 0 && (long long)(now_ns() - *ctl.t0) > ctl.timeout_ns) {
            flags[r] |= 4;
          } else if (!isfinite(res) || !isfinite(hn)) {
            flags[r] |= 1;
          } else if (res <= sc[3]) {
          } else if (hn <= brk * sqrt(colnorm2)) {
            flags[r] |= 2;
          } else if (it >= ctl.max_iters) {
          } else {
            stop = false;
          }
          if (stop) {
            active[r] = 0;
            break;
          }
        }
      }
    }
  } else if (lane == 0) {
    blkmask[r] = 0;
  }
  if (count_out != nullptr) {
    __shared__ int s_last;
    __threadfence();
    if (lane == 0) s_last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
    __syncwarp();
    if (s_last) {
      __threadfence();
      int cnt = 0;
      for (int q = lane; q < nrhs; q += 32) cnt += __ldcg(&active[q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
      if (lane == 0) {
        *count_out = cnt;
        *ticket = 0;
        if (ctl.graph) {
          const int jn = j + S;
          *ctl.jstep = jn;
          cudaGraphSetConditional(ctl.h_blk, (cnt > 0 && jn < *ctl.steps) ? 1u : 0u);
          *ctl.nlaunch += ctl.k_blk;
        }
      }
    }
  }
}


// Complex Givens rotation in FP32, the convention of givens():
// [c s; -conj(s) c] (a, b) = (rho, 0), c real.
__device__ __forceinline__ void givens_f(float2 a, float2 b, float& c, float2& s) {
  const float na = hypotf(a.x, a.y), nb = hypotf(b.x, b.y);
  if (nb == 0.f) {
    c = 1.f;
    s = make_float2(0.f, 0.f);
    return;
  }
  if (na == 0.f) {
    c = 0.f;
    s = make_float2(1.f, 0.f);
    return;
  }
  const float inr = rsqrtf(na * na + nb * nb);
  c = na * inr;
  const float2 ph = make_float2(a.x / na, a.y / na);
  s = make_float2((ph.x * b.x + ph.y * b.y) * inr, (ph.y * b.x - ph.x * b.y) * inr);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Newton shifts from the first cycle, one warp per right-hand side: the
// eigenvalues of the leading k x k block of the unrotated Hessenberg matrix,
// k = min(jlen, 4 S, 32), by shifted QR iterations in FP32 (the shifts only
// steer the conditioning of the Newton basis, so Ritz values to FP32
// accuracy serve; FP64 runs at 1/58 of the FP32 rate on this GPU): Wilkinson's
// shift, deflation when a subdiagonal entry falls below 4e-7 of its diagonal
// neighbours, at most 40 k iterations, after which the diagonal stands for
// the rest.  Then the first S of them in Leja order: the one of largest
// modulus, then each next maximising the product of its distances to those
// taken (Reichel 1990; ties to the lowest index).  Fewer than S Ritz values
// leave zero shifts.  Acts only at the end of the solve's first cycle
// (*scount, the cycles started, is 1; always when scount is null).
__global__ void __launch_bounds__(32)
    k_ritz(const double2* __restrict__ Hraw, const int* __restrict__ jlen,
           double2* __restrict__ theta, int S, int m, const int* __restrict__ scount) {
  pdl_entry();
  if (scount != nullptr && *scount != 1) return;
  __shared__ float2 A[32][33];
  __shared__ float2 rs[32];
  __shared__ float rc[32];
  __shared__ float2 ev[32];
  __shared__ int s_lo, s_hi, s_done;
  __shared__ float2 s_mu;
  const int r = blockIdx.x, lane = threadIdx.x;
  const int k = min(min(jlen[r], 4 * S), 32);
  const double2* hr = Hraw + (long)r * (m + 1) * m;
  for (int i = 0; i < k; ++i) {
    if (lane < k) {
      const double2 h = i <= lane + 1 ? hr[(long)lane * (m + 1) + i] : make_double2(0.0, 0.0);
      A[i][lane] = make_float2((float)h.x, (float)h.y);
    }
  }
  if (lane == 0) {
    s_hi = k - 1;
    s_done = 0;
  }
  __syncwarp();
  int iter = 0, since = 0;
  auto small = [&](int i) {  // A[i][i-1] negligible
    const float2 sub = A[i][i - 1];
    const float sc = hypotf(A[i][i].x, A[i][i].y) + hypotf(A[i - 1][i - 1].x, A[i - 1][i - 1].y);
    return hypotf(sub.x, sub.y) <= 4e-7f * sc;
  };
  while (true) {
    if (lane == 0) {
      int hi = s_hi;
      while (hi > 0 && small(hi)) {  // deflate at the bottom
        ev[hi] = A[hi][hi];
        --hi;
        since = 0;
      }
      if (hi == 0) ev[0] = A[0][0];
      const int done = hi <= 0 || iter >= 40 * k;
      if (done && hi > 0)
        for (int i = 0; i <= hi; ++i) ev[i] = A[i][i];
      int lo = hi;
      while (lo > 0) {
        if (small(lo)) {
          A[lo][lo - 1] = make_float2(0.f, 0.f);
          break;
        }
        --lo;
      }
      s_lo = lo;
      s_hi = hi;
      s_done = done;
      if (!done) {
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 nearer to its last entry
        const float2 a = A[hi - 1][hi - 1], b = A[hi - 1][hi], c = A[hi][hi - 1], d = A[hi][hi];
        const float2 h2 = make_float2(0.5f * (a.x - d.x), 0.5f * (a.y - d.y));
        const float2 hh = fmul2(h2, h2), bc = fmul2(b, c);
        const float2 disc2 = make_float2(hh.x + bc.x, hh.y + bc.y);
        const float mod = hypotf(disc2.x, disc2.y);
        const float sr = sqrtf(fmaxf(0.f, 0.5f * (mod + disc2.x)));
        float si = sqrtf(fmaxf(0.f, 0.5f * (mod - disc2.x)));
        if (disc2.y < 0.f) si = -si;
        const float2 mid = make_float2(0.5f * (a.x + d.x), 0.5f * (a.y + d.y));
        const float2 m1 = make_float2(mid.x + sr, mid.y + si), m2 = make_float2(mid.x - sr, mid.y - si);
        float2 mu = hypotf(m1.x - d.x, m1.y - d.y) <= hypotf(m2.x - d.x, m2.y - d.y) ? m1 : m2;
        if (since > 0 && since % 10 == 0) mu = make_float2(d.x + hypotf(c.x, c.y), d.y);  // exceptional
        s_mu = mu;
      }
    }
    __syncwarp();
    if (s_done) break;
    const int lo = s_lo, hi = s_hi;
    const float2 mu = s_mu;
    if (lane >= lo && lane <= hi) A[lane][lane] = make_float2(A[lane][lane].x - mu.x, A[lane][lane].y - mu.y);
    __syncwarp();
    // H - mu I = Q R by rotations of rows (kk, kk+1)
    for (int kk = lo; kk < hi; ++kk) {
      if (lane == 0) givens_f(A[kk][kk], A[kk + 1][kk], rc[kk], rs[kk]);
      __syncwarp();
      const float c = rc[kk];
      const float2 s = rs[kk];
      if (lane >= kk && lane <= hi) {
        const float2 x = A[kk][lane], y = A[kk + 1][lane];
        A[kk][lane] = make_float2(c * x.x + (s.x * y.x - s.y * y.y), c * x.y + (s.x * y.y + s.y * y.x));
        A[kk + 1][lane] = make_float2(-(s.x * x.x + s.y * x.y) + c * y.x, -(s.x * x.y - s.y * x.x) + c * y.y);
      }
      __syncwarp();
    }
    // R Q: columns (kk, kk+1) times G^H = [[c, -s], [conj(s), c]]
    for (int kk = lo; kk < hi; ++kk) {
      const float c = rc[kk];
      const float2 s = rs[kk];
      if (lane >= lo && lane <= min(kk + 1, hi)) {
        const float2 x = A[lane][kk], y = A[lane][kk + 1];
        A[lane][kk] = make_float2(c * x.x + (y.x * s.x + y.y * s.y), c * x.y + (y.y * s.x - y.x * s.y));
        A[lane][kk + 1] = make_float2(-(x.x * s.x - x.y * s.y) + c * y.x, -(x.x * s.y + x.y * s.x) + c * y.y);
      }
      __syncwarp();
    }
    if (lane >= lo && lane <= hi) A[lane][lane] = make_float2(A[lane][lane].x + mu.x, A[lane][lane].y + mu.y);
    __syncwarp();
    ++iter;
    ++since;
  }
  // Leja order of ev[0..k-1]; lanes over the candidates
  const float2 z = lane < k ? ev[lane] : make_float2(0.f, 0.f);
  float score = lane < k ? hypotf(z.x, z.y) : -INFINITY;
  bool taken = false;
  for (int t = 0; t < S; ++t) {
    float best = (lane < k && !taken) ? score : -INFINITY;
    int who = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int ow = __shfl_xor_sync(0xffffffffu, who, o);
      if (ob > best || (ob == best && ow < who)) {
        best = ob;
        who = ow;
      }
    }
    const float2 zc = make_float2(__shfl_sync(0xffffffffu, z.x, who), __shfl_sync(0xffffffffu, z.y, who));
    if (lane == 0)
      theta[(long)r * kSMax + t] = t < k ? make_double2(zc.x, zc.y) : make_double2(0.0, 0.0);
    if (lane == who) taken = true;
    // from now on the score is the log of the product of distances
    score = (t == 0 ? 0.f : score) + logf(hypotf(z.x - zc.x, z.y - zc.y));
  }
  if (lane == 0)
    for (int t = S; t < kSMax; ++t) theta[(long)r * kSMax + t] = make_double2(0.0, 0.0);
}
