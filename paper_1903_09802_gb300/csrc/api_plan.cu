// Plan creation: workspace layout, Green-function spectrum, polarizabilities,
// incident field and the standalone 3-D FFT entry point.
#include <atomic>
#include <cstdlib>
#include <cmath>
#include <complex>
#include <cstring>
#include <string>

#include "fft_kernels.cuh"
#include "plan.hpp"

namespace dda {

namespace {
thread_local std::string g_err;
std::atomic<long long> g_launches{0};
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_counter() { return g_launches.load(std::memory_order_relaxed); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool solve_graph_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("DDA_SOLVE_GRAPH");
    return !(e && e[0] == '0');
  }();
  return on;
}

void set_error(const std::string& msg) { g_err = msg; }

dda_status_t fail(dda_status_t st, const std::string& msg) {
  g_err = msg;
  return st;
}

dda_status_t check_cuda(const char* where) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(DDA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
  return DDA_OK;
}

namespace {

constexpr double kPi = 3.14159265358979323846;

bool valid_desc(const dda_plan_desc_t& d, std::string& why, dda_status_t& st) {
  st = DDA_ERR_INVALID_ARG;
  if (d.l < 1 || d.m < 1 || d.n < 1) return why = "box edges must be >= 1", false;
  if (!(d.dx > 0) || !(d.k > 0) || !std::isfinite(d.dx) || !std::isfinite(d.k))
    return why = "dx and k must be positive and finite", false;
  if (d.n_materials < 1 || d.n_materials > 255) return why = "n_materials must be 1..255", false;
  if (d.max_rhs < 1 || d.max_rhs > 4096) return why = "max_rhs must be 1..4096", false;
  if (d.krylov_m < 0 || d.krylov_m > 512) return why = "krylov_m must be 0..512", false;
  if (d.precond2 < 0 || d.precond2 > 3)
    return why = "precond2 must be 0 (none) or 1, 2, 3 (Toeplitz level z, x, y)", false;
  if (d.circulant != 0 && d.circulant != 1) return why = "circulant must be 0 (Chan) or 1 (Strang)", false;
  if (d.voxel_eps != 0 && d.voxel_eps != 1) return why = "voxel_eps must be 0 or 1", false;
  if (d.rhs_chunk < 0) return why = "rhs_chunk must be >= 0", false;
  if (d.krylov_c64 != 0 && d.krylov_c64 != 1) return why = "krylov_c64 must be 0 or 1", false;
  if (d.krylov_c64 && !(d.precisions & DDA_PLAN_C64))
    return why = "krylov_c64 needs a plan holding complex64 data", false;
  if (d.sstep != 0 && (d.sstep < 2 || d.sstep > 8))
    return why = "sstep must be 0 or 2..8", false;
  if (d.sstep > d.krylov_m) return why = "sstep must be at most krylov_m", false;
  if ((d.precisions & (DDA_PLAN_C128 | DDA_PLAN_C64)) == 0 ||
      (d.precisions & ~(DDA_PLAN_C128 | DDA_PLAN_C64)) != 0)
    return why = "precisions must be a non-empty set of DDA_PLAN_C128 | DDA_PLAN_C64", false;
  st = DDA_ERR_UNSUPPORTED_SIZE;
  for (int e : {d.l, d.m, d.n}) {
    if (e > 512)
      return why = "box edges must be at most 512", false;
    // mixed-radix transforms: even 7-smooth edges (radices 2, 4, 3, 5, 7)
    if (!is_pow2(e) && !(e % 2 == 0 && is_7smooth(e) && make_radix_plan(e).nst > 0 &&
                         make_radix_plan(2 * e).nst > 0))
      return why = "box edges must be powers of two or even 7-smooth numbers (2^a 3^b 5^c 7^d)",
             false;
    // the mixed-radix three-component tile of lengths e and 2e (8 values per
    // thread, a power-of-two column count that makes the values a multiple of
    // 8) must fit the double-float kernel's 256 threads
    if (!is_pow2(e))
      for (long L : {(long)e, 2L * e}) {
        long nb = 1;
        while ((3 * nb * L) % 8 != 0) nb *= 2;
        if (3 * nb * L / 8 > 256)
          return why = "mixed-radix edge " + std::to_string(e) +
                       " needs a transform tile above 256 threads (every even 7-smooth edge up "
                       "to 208 is taken)",
                 false;
      }
  }
  if (twiddle_length(d.l, d.m, d.n) > kMaxTwiddleLength)
    return why = "the least common multiple of the padded edges 2l, 2m, 2n must be at most 2^20",
           false;
  st = DDA_OK;
  return true;
}

}  // namespace

bool make_layout(const dda_plan_desc_t& d, void* ws, Layout& L, std::string& why) {
  dda_status_t st;
  if (!valid_desc(d, why, st)) return false;
  Carver c(ws);
  const long l = d.l, m = d.m, n = d.n;
  const long Lx = 2 * l, Ly = 2 * m, Lz = 2 * n;
  const long nvox = l * m * n, P = Lx * Ly * Lz;
  const long Lmax = twiddle_length(l, m, n);
  const bool h128 = d.precisions & DDA_PLAN_C128, h64 = d.precisions & DDA_PLAN_C64;
  const size_t esz = h128 ? 16 : 8;
  const long gsz = (l + 1) * (m + 1) * (n + 1) * 6;
  const long csz = (l / 2 + 1) * (m / 2 + 1) * (n / 2 + 1) * 6;
  const long R = d.max_rhs, K1 = d.n_materials + 1;
  const long nu = 3 * nvox;
  L.tw128 = c.take(Lmax * 16);
  L.tw64 = c.take(Lmax * 8);
  if (h128) {
    L.G128 = c.take(gsz * 16);
    L.C128 = c.take(csz * 16);
    L.twdf = c.take(Lmax * 16);
    L.Gdf = c.take(gsz * 16);
    L.ainvdf = c.take(R * K1 * 16);
  }
  if (h64) {
    L.G64 = c.take(gsz * 8);
    L.C64 = c.take(csz * 8);
  }
  L.ainv128 = c.take(R * K1 * 16);
  L.ainv64 = c.take(R * K1 * 8);
  L.incd = static_cast<double*>(c.take(R * 6 * sizeof(double)));
  if (d.voxel_eps) {
    L.eps_vox = c.take(16 * nvox);
    L.pv128 = c.take(16 * R * nvox);
    L.pv64 = c.take(8 * R * nvox);
    if (h128) L.pvdf = c.take(16 * R * nvox);
  }
  L.dainv128 = c.take(R * K1 * 16);
  // FFT scratch for one chunk of right-hand sides
  const long RC = d.rhs_chunk > 0 ? std::min<long>(d.rhs_chunk, R) : R;
  // (its head also holds the cross sections' block sums: 4 doubles per block
  // of at most 304, per right-hand side)
  const size_t xsec = (size_t)32 * std::min<long>(304, std::max<long>(1, (nvox + 4095) / 4096)) * R;
  L.buf1 = c.take(std::max<size_t>(esz * RC * 3 * n * m * Lx, xsec));
  size_t b2 = esz * RC * 3 * n * Ly * Lx;
  b2 = std::max(b2, (size_t)P * 16);     // Green-function spectrum build (complex128)
  b2 = std::max(b2, (size_t)nvox * 96);  // circulant build: six complex128 components
  L.buf2 = c.take(b2);
  L.err_flag = c.take(64);
  if (d.precond2) {
    // edges of the relabelled box whose z is the Toeplitz level
    const long fl = d.precond2 == 2 ? m : (d.precond2 == 3 ? n : l);
    const long fm = d.precond2 == 2 ? n : (d.precond2 == 3 ? l : m);
    const long fn = d.precond2 == 2 ? l : (d.precond2 == 3 ? m : n);
    L.P2 = c.take((size_t)(fl / 2 + 1) * (fm / 2 + 1) * (3 * fn) * (3 * fn) * 8);
    L.C2 = c.take((size_t)6 * (2 * fn - 1) * fl * fm * 16);
    if (d.precond2 != 1) L.mat2 = c.take(nvox);
  }
  // complex128 field batch: the solver's residual and the cross sections' A c
  if (h128) L.R128 = c.take(16 * R * nu);
  if (d.krylov_m > 0) {
    const long mk = d.krylov_m;
    // Gram-Schmidt reduction blocks per right-hand side: at most one wave of
    // 3 blocks x 152 SMs, chunks of at least 512 values
    L.nblk = (int)std::min<long>(456, std::max<long>(1, (nu + 511) / 512));
    // basis and step vectors in the inner precision: complex64 only when the
    // plan is limited to complex64 cycles (krylov_c64)
    const size_t vsz = d.krylov_c64 ? 8 : esz;
    L.V = c.take(vsz * (mk + 1) * R * nu);
    L.Wv = c.take(vsz * R * nu);
    L.Zv = c.take(vsz * R * nu);
    L.B128 = c.take(16 * R * nu);
    SolverState& s = L.st;
    s.H = static_cast<double2*>(c.take(16 * R * (mk + 1) * mk));
    s.cs = static_cast<double*>(c.take(8 * R * mk));
    s.sn = static_cast<double2*>(c.take(16 * R * mk));
    s.g = static_cast<double2*>(c.take(16 * R * (mk + 1)));
    s.y = static_cast<double2*>(c.take(16 * R * mk));
    s.hcol = static_cast<double2*>(c.take(16 * R * (mk + 2)));
    s.partial = static_cast<double2*>(c.take(16 * R * (size_t)L.nblk * (mk + 2)));
    s.scal = static_cast<double*>(c.take(8 * R * 16));
    s.active = static_cast<int*>(c.take(4 * R));
    s.jlen = static_cast<int*>(c.take(4 * R));
    s.flags = static_cast<int*>(c.take(4 * R));
    s.iters = static_cast<int*>(c.take(4 * R));
    s.run = static_cast<int*>(c.take(4 * R));
    s.reorth = static_cast<int*>(c.take(4 * R));
    s.reorth_count = static_cast<int*>(c.take(4 * R));
    s.tickets = static_cast<int*>(c.take(8 * R));
    s.bscal = static_cast<double*>(c.take(8 * 16 * R));
    s.counters = static_cast<int*>(c.take(64));
    s.ctl = static_cast<int*>(c.take(16));
    s.out = c.take((size_t)kRhsOutBytes * R);
    s.hist = static_cast<double*>(c.take(sizeof(double) * kHistCap * R));
    s.t0 = static_cast<unsigned long long*>(c.take(8));
    s.nlaunch = static_cast<long long*>(c.take(8));
    if (d.sstep > 0) {
      const long sb = d.sstep;
      L.Wb = c.take(vsz * sb * R * nu);
      s.Hraw = static_cast<double2*>(c.take(16 * R * (mk + 1) * mk));
      s.theta = static_cast<double2*>(c.take(16 * R * 8));
      s.cb = static_cast<double2*>(c.take(16 * R * 2 * (mk + 1 + sb) * sb));
      s.rinv = static_cast<double2*>(c.take(16 * R * 64));
      // block dot partials: nrhs * max(ceil(304 / nrhs), ceil(nu s / 8192)) blocks
      const long nbmax = 304 + R + R * ((nu * sb + 8191) / 8192);
      s.bpart = static_cast<double2*>(c.take(16 * nbmax * (mk + 1 + sb) * sb));
    }
  }
  L.total = c.off + 256;
  return true;
}

namespace {

// One component of g(R) (the Green function of Section 2, in the form of
// Algorithm 1) in FP64.
__device__ __forceinline__ double2 green_component(double X, double Y, double Z, double k, int a,
                                                   int b) {
  const double r2 = X * X + Y * Y + Z * Z;
  const double r = sqrt(r2);
  const double rv[3] = {X / r, Y / r, Z / r};
  double sn, cs;
  sincos(k * r, &sn, &cs);
  const double er = cs / r, ei = sn / r;  // e^{ikr} / r
  const double dlt = (a == b) ? 1.0 : 0.0;
  const double pp = rv[a] * rv[b];
  const double q = (dlt - 3.0 * pp) / r2;
  const double br = k * k * (dlt - pp) - q;  // k^2 (d - pp) + (i k r - 1)(d - 3pp)/r^2
  const double bi = k * r * q;
  return make_double2(er * br - ei * bi, er * bi + ei * br);
}

__device__ const int kCompA[6] = {0, 0, 0, 1, 1, 2};
__device__ const int kCompB[6] = {0, 1, 2, 1, 2, 2};

// Index p of a padded axis of length Lp >= 2l - 1 as a signed voxel offset:
// p < l -> p, p > Lp - l -> p - Lp, otherwise the wrap region (no pair of
// box voxels has that offset), reported invalid.
__device__ __forceinline__ bool padded_offset(long p, long l, long Lp, long& o) {
  if (p < l) {
    o = p;
    return true;
  }
  if (p > Lp - l) {
    o = p - Lp;
    return true;
  }
  return false;
}

// Circulant generator of component c on the padded grid (Section 2.2: the
// BTTB block is embedded in a circulant of twice the size per level).
__global__ void k_green_generator(double2* out, int c, long l, long m, long n, long Lx, long Ly,
                                  long Lz, double dx, double k) {
  pdl_entry();
  const long P = Lx * Ly * Lz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < P;
       i += (long)gridDim.x * blockDim.x) {
    const long x = i % Lx, y = (i / Lx) % Ly, z = i / (Lx * Ly);
    long ox, oy, oz;
    double2 v = make_double2(0.0, 0.0);
    if (padded_offset(x, l, Lx, ox) && padded_offset(y, m, Ly, oy) && padded_offset(z, n, Lz, oz) &&
        (ox | oy | oz) != 0)
      v = green_component(dx * ox, dx * oy, dx * oz, k, kCompA[c], kCompB[c]);
    out[i] = v;
  }
}

// Keep the octant 0..L/2 of each axis of a full spectrum (the rest follows
// from the block's parity) as component c.  The complex128 store interleaves
// the six components of a frequency ([z][y][x][6]); the complex64 store keeps
// them as three planes of component pairs per (z, y) row,
// [z][y][pair c/2][x][c%2], so that the 16-byte pair loads of neighbouring x
// frequencies are contiguous (one 128-byte line for 8 frequencies).
__global__ void k_compress(const double2* full, long Lx, long Ly, long Lz, long hx, long hy,
                           long hz, int c, double2* out128, float2* out64) {
  pdl_entry();
  const long H = hx * hy * hz;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < H;
       i += (long)gridDim.x * blockDim.x) {
    const long x = i % hx, y = (i / hx) % hy, z = i / (hx * hy);
    const double2 v = full[(z * Ly + y) * Lx + x];
    if (out128) out128[i * 6 + c] = v;
    if (out64)
      out64[(((z * hy + y) * 3 + c / 2) * hx + x) * 2 + (c & 1)] =
          make_float2((float)v.x, (float)v.y);
  }
}

// E_inc = pol exp(i k dir . r) on scatterer voxels, r from the box centre.
__global__ void k_incident(double2* b, const uint8_t* mat, const double* inc, int nrhs, long l,
                           long m, long n, double dx, double k, double sgn) {
  pdl_entry();
  const long nvox = l * m * n;
  const long tot = nvox * nrhs;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    const long v = i % nvox, r = i / nvox;
    const long x = v % l, y = (v / l) % m, z = v / (l * m);
    const double* d = inc + r * 6;
    double2 out[3] = {{0, 0}, {0, 0}, {0, 0}};
    if (mat[v] != 0) {
      const double px = dx * (x - 0.5 * (l - 1)), py = dx * (y - 0.5 * (m - 1)),
                   pz = dx * (z - 0.5 * (n - 1));
      double sn, cs;
      sincos(k * (d[0] * px + d[1] * py + d[2] * pz), &sn, &cs);
      for (int c = 0; c < 3; ++c) out[c] = make_double2(d[3 + c] * cs, sgn * d[3 + c] * sn);
    }
    for (int c = 0; c < 3; ++c) b[(r * 3 + c) * nvox + v] = out[c];
  }
}

inline unsigned grid_for(long n, int threads) {
  const long g = (n + threads - 1) / threads;
  return (unsigned)std::min<long>(std::max<long>(g, 1), 152L * 32);
}

}  // namespace

}  // namespace dda

using namespace dda;

extern "C" const char* dda_last_error(void) { return g_err.c_str(); }

extern "C" int64_t dda_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" size_t dda_workspace_size(const dda_plan_desc_t* desc) {
  if (!desc) {
    set_error("dda_workspace_size: desc is NULL");
    return 0;
  }
  Layout L;
  std::string why;
  if (!make_layout(*desc, nullptr, L, why)) {
    set_error("dda_workspace_size: " + why);
    return 0;
  }
  return L.total;
}

namespace dda {
namespace {

__device__ __forceinline__ double2 cdivd(double2 a, double2 b) {
  const double dn = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / dn, (a.y * b.x - a.x * b.y) / dn);
}

// alpha^{-1} of every scatterer voxel for every right-hand side from the
// voxel's own permittivity: 1/alpha = 1/alpha_CM + (b1 + eps b2 + eps b3 S)(k dx)^2
// - (2i/3)(k dx)^3 with 1/alpha_CM = (4 pi/3)(eps + 2)/(eps - 1) (Section 2.1,
// the LDR display), S = sum_j (d_j e_j)^2 of the right-hand side's wave.
// Air voxels get alpha_tilde^{-1} (ainv[rhs][0]); they are never read.
__global__ void k_voxel_ainv(const double2* __restrict__ eps, const uint8_t* __restrict__ mat,
                             const double* __restrict__ incd, const double2* __restrict__ ainv,
                             int K1, int nrhs, long nvox, double kd, double2* __restrict__ pv128,
                             float2* __restrict__ pv64, cx<df>* __restrict__ pvdf,
                             int* __restrict__ err) {
  pdl_entry();
  const double pi = 3.14159265358979323846;
  const long tot = nvox * nrhs;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < tot;
       i += (long)gridDim.x * blockDim.x) {
    const long v = i % nvox;
    const int r = (int)(i / nvox);
    double2 a = ainv[(long)r * K1];
    if (mat[v] != 0) {
      const double2 e = eps[v];
      const double* q = incd + r * 6;
      double S = 0.0;
      for (int c = 0; c < 3; ++c) S += (q[c] * q[3 + c]) * (q[c] * q[3 + c]);
      const double2 cm = cdivd(make_double2(e.x + 2.0, e.y), make_double2(e.x - 1.0, e.y));
      const double b = -1.7700004 * S + 0.1648469;
      const double kd2 = kd * kd;
      a.x = (4.0 * pi / 3.0) * cm.x + (-1.891531 + e.x * b) * kd2;
      a.y = (4.0 * pi / 3.0) * cm.y + e.y * b * kd2 - (2.0 / 3.0) * kd2 * kd;
      if (!isfinite(a.x) || !isfinite(a.y)) atomicOr(err, 2);
    }
    pv128[i] = a;
    pv64[i] = make_float2((float)a.x, (float)a.y);
    if (pvdf != nullptr) pvdf[i] = mk<df>(df(a.x), df(a.y));
  }
}

// Tabulate the per-voxel polarizabilities for the current incidences.
dda_status_t tabulate_voxel_ainv(dda_plan_s* p, cudaStream_t s) {
  if (!p->voxel_eps_on || p->nrhs_inc < 1) return DDA_OK;
  cudaMemsetAsync(p->w.err_flag, 0, 4, s);
  const long tot = p->nvox * p->nrhs_inc;
  const unsigned grid = (unsigned)std::min<long>(std::max<long>((tot + 255) / 256, 1), 152L * 32);
  note_launch();
  k_voxel_ainv<<<grid, 256, 0, s>>>(
      static_cast<const double2*>(p->w.eps_vox), p->mat, p->w.incd,
      static_cast<const double2*>(p->w.ainv128), p->K + 1, p->nrhs_inc, p->nvox,
      p->d.k * p->d.dx, static_cast<double2*>(p->w.pv128), static_cast<float2*>(p->w.pv64),
      static_cast<cx<df>*>(p->w.pvdf), static_cast<int*>(p->w.err_flag));
  int err = 0;
  cudaMemcpyAsync(&err, p->w.err_flag, 4, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) return check_cuda("dda_set_voxel_eps");
  if (err) return fail(DDA_ERR_INVALID_ARG, "dda_set_voxel_eps: a voxel's polarizability is "
                                            "singular (eps = 1 on a scatterer voxel?)");
  return DDA_OK;
}

}  // namespace
}  // namespace dda

extern "C" dda_status_t dda_plan_create(dda_plan_t* out, const dda_plan_desc_t* desc,
                                        const uint8_t* d_mat, const double* h_eps, void* d_work,
                                        size_t work_bytes, void* stream) {
  if (!out || !desc || !d_mat || !h_eps || !d_work)
    return fail(DDA_ERR_INVALID_ARG, "dda_plan_create: NULL argument");
  *out = nullptr;
  std::string why;
  dda_status_t st;
  if (!valid_desc(*desc, why, st)) return fail(st, "dda_plan_create: " + why);
  if (reinterpret_cast<uintptr_t>(d_work) % 256 != 0)
    return fail(DDA_ERR_WORKSPACE, "dda_plan_create: workspace must be 256-byte aligned");
  Layout L;
  make_layout(*desc, d_work, L, why);
  if (work_bytes < L.total)
    return fail(DDA_ERR_WORKSPACE, "dda_plan_create: workspace of " + std::to_string(work_bytes) +
                                       " bytes, need " + std::to_string(L.total));
  for (int i = 0; i < 2 * desc->n_materials; ++i)
    if (!std::isfinite(h_eps[i])) return fail(DDA_ERR_INVALID_ARG, "dda_plan_create: eps not finite");
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  dda_plan_s* p = new dda_plan_s();
  static std::atomic<long long> next_id{1};
  p->id = next_id.fetch_add(1);
  p->d = *desc;
  p->l = desc->l;
  p->m = desc->m;
  p->n = desc->n;
  p->Lx = 2 * p->l;
  p->Ly = 2 * p->m;
  p->Lz = 2 * p->n;
  p->Lmax = (int)twiddle_length(p->l, p->m, p->n);
  p->nvox = (long)p->l * p->m * p->n;
  p->P = (long)p->Lx * p->Ly * p->Lz;
  p->hx = p->l + 1;
  p->hy = p->m + 1;
  p->hz = p->n + 1;
  p->cx_ = p->l / 2 + 1;
  p->cy_ = p->m / 2 + 1;
  p->cz_ = p->n / 2 + 1;
  p->K = desc->n_materials;
  p->rhs_chunk = desc->rhs_chunk > 0 ? std::min(desc->rhs_chunk, desc->max_rhs) : desc->max_rhs;
  p->mat = d_mat;
  p->eps.assign(h_eps, h_eps + 2 * desc->n_materials);
  p->w = L;
  p->has128 = desc->precisions & DDA_PLAN_C128;
  p->has64 = desc->precisions & DDA_PLAN_C64;

  // material census (alpha_tilde is the most frequent non-air material)
  std::vector<uint8_t> hm(p->nvox);
  cudaMemcpyAsync(hm.data(), d_mat, p->nvox, cudaMemcpyDeviceToHost, s);
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    delete p;
    return check_cuda("dda_plan_create: reading materials");
  }
  p->mat_count.assign(p->K + 1, 0);
  for (uint8_t v : hm) {
    if (v > p->K) {
      delete p;
      return fail(DDA_ERR_INVALID_ARG, "dda_plan_create: material index above n_materials");
    }
    p->mat_count[v]++;
  }

  // twiddles exp(-2 pi i t / Lmax)
  {
    std::vector<double2> t128(p->Lmax);
    std::vector<float2> t64(p->Lmax);
    for (int t = 0; t < p->Lmax; ++t) {
      const double a = -2.0 * kPi * (double)t / (double)p->Lmax;
      t128[t] = make_double2(std::cos(a), std::sin(a));
      t64[t] = make_float2((float)t128[t].x, (float)t128[t].y);
    }
    cudaMemcpyAsync(L.tw128, t128.data(), p->Lmax * 16, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(L.tw64, t64.data(), p->Lmax * 8, cudaMemcpyHostToDevice, s);
    if (L.twdf) {
      std::vector<cx<df>> tdf(p->Lmax);
      for (int t = 0; t < p->Lmax; ++t) tdf[t] = mk<df>(df(t128[t].x), df(t128[t].y));
      cudaMemcpyAsync(L.twdf, tdf.data(), p->Lmax * 16, cudaMemcpyHostToDevice, s);
    }
  }
  cudaMemsetAsync(L.err_flag, 0, 64, s);

  // kernel spectrum, one component at a time through the FP64 scratch
  double2* scratch = static_cast<double2*>(L.buf2);
  for (int c = 0; c < 6; ++c) {
    note_launch();
    k_green_generator<<<grid_for(p->P, 256), 256, 0, s>>>(scratch, c, p->l, p->m, p->n, p->Lx, p->Ly,
                                                          p->Lz, desc->dx, desc->k);
    fft3d_inplace<double, false>(reinterpret_cast<cx<double>*>(scratch), 1, p->Lx, p->Ly, p->Lz, 1.0,
                                 static_cast<const cx<double>*>(L.tw128), p->Lmax, s);
    note_launch();
    k_compress<<<grid_for((long)p->hx * p->hy * p->hz, 256), 256, 0, s>>>(
        scratch, p->Lx, p->Ly, p->Lz, p->hx, p->hy, p->hz, c, static_cast<double2*>(L.G128),
        static_cast<float2*>(L.G64));
  }
  if (L.Gdf) {
    const long ng = (long)p->hx * p->hy * p->hz * 6;
    note_launch();
    k_to_df<<<grid_for(ng, 256), 256, 0, s>>>(static_cast<const double2*>(L.G128),
                                                static_cast<cx<df>*>(L.Gdf), ng);
  }
  dda_status_t cs = check_cuda("dda_plan_create");
  if (cs == DDA_OK) cs = noalloc_prepare();
  if (cs != DDA_OK) {
    delete p;
    return cs;
  }
  *out = p;
  return DDA_OK;
}

extern "C" dda_status_t dda_set_incidence(dda_plan_t p, int32_t nrhs, const dda_incidence_t* inc,
                                          void* stream) {
  if (!p || !inc) return fail(DDA_ERR_INVALID_ARG, "dda_set_incidence: NULL argument");
  if (nrhs < 1 || nrhs > p->d.max_rhs)
    return fail(DDA_ERR_INVALID_ARG, "dda_set_incidence: nrhs outside 1..max_rhs");
  const int K1 = p->K + 1;
  std::vector<double> h(nrhs * 6);
  p->ainv_host.assign((size_t)nrhs * K1 * 2, 0.0);
  p->ainv_host32.assign((size_t)nrhs * K1 * 2, 0.0f);
  p->dainv_host.assign((size_t)nrhs * K1 * 2, 0.0);
  // most frequent non-air material, ties to the lowest index
  int tilde = 1;
  for (int mt = 2; mt <= p->K; ++mt)
    if (p->mat_count[mt] > p->mat_count[tilde]) tilde = mt;
  const double kd = p->d.k * p->d.dx;
  for (int r = 0; r < nrhs; ++r) {
    const double* d = inc[r].dir;
    const double* e = inc[r].pol;
    const double nd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double ne = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const double de = d[0] * e[0] + d[1] * e[1] + d[2] * e[2];
    if (!(std::fabs(nd - 1) < 1e-9 && std::fabs(ne - 1) < 1e-9 && std::fabs(de) < 1e-9))
      return fail(DDA_ERR_INVALID_ARG, "dda_set_incidence: dir and pol must be orthonormal");
    for (int c = 0; c < 3; ++c) {
      h[r * 6 + c] = d[c];
      h[r * 6 + 3 + c] = e[c];
    }
    // S = sum_j (d_j e_j)^2 (Section 2.1)
    double S = 0;
    for (int c = 0; c < 3; ++c) S += (d[c] * e[c]) * (d[c] * e[c]);
    std::vector<std::complex<double>> ainv(K1);
    for (int mt = 1; mt <= p->K; ++mt) {
      const std::complex<double> eps(p->eps[2 * (mt - 1)], p->eps[2 * (mt - 1) + 1]);
      // Clausius-Mossotti and the lattice dispersion relation (Section 2.1)
      const std::complex<double> acm = 3.0 / (4.0 * kPi) * (eps - 1.0) / (eps + 2.0);
      const std::complex<double> corr =
          (-1.891531 + eps * 0.1648469 + eps * (-1.7700004) * S) * (kd * kd) -
          std::complex<double>(0.0, 2.0 / 3.0) * (kd * kd * kd);
      const std::complex<double> alpha = acm / (1.0 + acm * corr);
      ainv[mt] = 1.0 / alpha;
      // d(1/alpha)/d(eps): 1/alpha = (4 pi/3)(eps+2)/(eps-1) + corr(eps)
      const std::complex<double> dinv =
          -4.0 * kPi / ((eps - 1.0) * (eps - 1.0)) + (0.1648469 + (-1.7700004) * S) * (kd * kd);
      p->dainv_host[(r * K1 + mt) * 2] = dinv.real();
      p->dainv_host[(r * K1 + mt) * 2 + 1] = dinv.imag();
    }
    ainv[0] = ainv[tilde];  // air rows and the preconditioner use alpha_tilde
    for (int mt = 0; mt < K1; ++mt) {
      if (!std::isfinite(ainv[mt].real()) || !std::isfinite(ainv[mt].imag()))
        return fail(DDA_ERR_INVALID_ARG,
                    "dda_set_incidence: polarizability is zero or singular (eps = 1 or -2?)");
      p->ainv_host[(r * K1 + mt) * 2] = ainv[mt].real();
      p->ainv_host[(r * K1 + mt) * 2 + 1] = ainv[mt].imag();
      p->ainv_host32[(r * K1 + mt) * 2] = (float)ainv[mt].real();
      p->ainv_host32[(r * K1 + mt) * 2 + 1] = (float)ainv[mt].imag();
    }
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemcpyAsync(p->w.incd, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(p->w.ainv128, p->ainv_host.data(), p->ainv_host.size() * sizeof(double),
                  cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(p->w.ainv64, p->ainv_host32.data(), p->ainv_host32.size() * sizeof(float),
                  cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(p->w.dainv128, p->dainv_host.data(), p->dainv_host.size() * sizeof(double),
                  cudaMemcpyHostToDevice, s);
  if (p->w.ainvdf) {
    std::vector<cx<df>> adf(p->ainv_host.size() / 2);
    for (size_t i = 0; i < adf.size(); ++i)
      adf[i] = mk<df>(df(p->ainv_host[2 * i]), df(p->ainv_host[2 * i + 1]));
    cudaMemcpyAsync(p->w.ainvdf, adf.data(), adf.size() * 16, cudaMemcpyHostToDevice, s);
  }
  p->inc.assign(inc, inc + nrhs);
  p->nrhs_inc = nrhs;
  const dda_status_t st = check_cuda("dda_set_incidence");
  if (st != DDA_OK) return st;
  return tabulate_voxel_ainv(p, s);
}

extern "C" dda_status_t dda_set_voxel_eps(dda_plan_t p, const void* d_eps, void* stream) {
  if (!p) return fail(DDA_ERR_INVALID_ARG, "dda_set_voxel_eps: NULL plan");
  if (!p->d.voxel_eps)
    return fail(DDA_ERR_INVALID_ARG, "dda_set_voxel_eps: plan made without voxel_eps");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (d_eps == nullptr) {
    p->voxel_eps_on = false;
    return DDA_OK;
  }
  cudaMemcpyAsync(p->w.eps_vox, d_eps, 16 * p->nvox, cudaMemcpyDeviceToDevice, s);
  p->voxel_eps_on = true;
  dda_status_t st = check_cuda("dda_set_voxel_eps");
  if (st == DDA_OK) st = tabulate_voxel_ainv(p, s);
  if (st != DDA_OK) p->voxel_eps_on = false;
  return st;
}

extern "C" dda_status_t dda_incident_field(dda_plan_t p, int32_t nrhs, void* d_b, void* stream) {
  if (!p || !d_b) return fail(DDA_ERR_INVALID_ARG, "dda_incident_field: NULL argument");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_incident_field: nrhs above the incidence count set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  note_launch();
  k_incident<<<grid_for(p->nvox * nrhs, 256), 256, 0, s>>>(static_cast<double2*>(d_b), p->mat,
                                                          p->w.incd, nrhs, p->l, p->m, p->n,
                                                          p->d.dx, p->d.k, 1.0);
  return check_cuda("dda_incident_field");
}

extern "C" dda_status_t dda_adjoint_rhs(dda_plan_t p, int32_t nrhs, void* d_b, void* stream) {
  if (!p || !d_b) return fail(DDA_ERR_INVALID_ARG, "dda_adjoint_rhs: NULL argument");
  if (nrhs < 1 || nrhs > p->nrhs_inc)
    return fail(DDA_ERR_INVALID_ARG, "dda_adjoint_rhs: nrhs above the incidence count set");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  note_launch();
  k_incident<<<grid_for(p->nvox * nrhs, 256), 256, 0, s>>>(static_cast<double2*>(d_b), p->mat,
                                                          p->w.incd, nrhs, p->l, p->m, p->n,
                                                          p->d.dx, p->d.k, -1.0);
  return check_cuda("dda_adjoint_rhs");
}

extern "C" dda_status_t dda_fft3d(dda_plan_t p, int32_t prec, int32_t nbatch, void* d_data,
                                  int32_t inverse, void* stream) {
  if (!p || !d_data) return fail(DDA_ERR_INVALID_ARG, "dda_fft3d: NULL argument");
  if (nbatch < 1) return fail(DDA_ERR_INVALID_ARG, "dda_fft3d: nbatch must be >= 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const double sc = inverse ? 1.0 / (double)p->nvox : 1.0;
  if (prec == DDA_C128) {
    auto* d = static_cast<cx<double>*>(d_data);
    if (inverse)
      fft3d_inplace<double, true>(d, nbatch, p->l, p->m, p->n, sc, tw_of<double>(p), p->Lmax, s);
    else
      fft3d_inplace<double, false>(d, nbatch, p->l, p->m, p->n, 1.0, tw_of<double>(p), p->Lmax, s);
  } else if (prec == DDA_C64) {
    auto* d = static_cast<cx<float>*>(d_data);
    if (inverse)
      fft3d_inplace<float, true>(d, nbatch, p->l, p->m, p->n, (float)sc, tw_of<float>(p), p->Lmax, s);
    else
      fft3d_inplace<float, false>(d, nbatch, p->l, p->m, p->n, 1.0f, tw_of<float>(p), p->Lmax, s);
  } else {
    return fail(DDA_ERR_INVALID_ARG, "dda_fft3d: prec must be DDA_C128 or DDA_C64");
  }
  return check_cuda("dda_fft3d");
}

extern "C" void dda_plan_destroy(dda_plan_t p) {
  if (!p) return;
  if (p->pinned) cudaFreeHost(p->pinned);
  delete p;
}
