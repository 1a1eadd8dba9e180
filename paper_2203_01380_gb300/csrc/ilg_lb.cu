// Lattice Boltzmann comparator (Sec. IV, Eq. MRTLB) in double precision.
//
// With one rate omega^j for the odd (current) moments and one rate omega for the
// even non-conserved ones, the moment-space update splits by parity: the part of
// f - f^0 that is odd under v -> -v is exactly its projection on the odd moments,
// the even part its projection on the even ones (the transform matrix is
// orthonormal under the symmetric weights and every moment has a definite parity).
// So, per opposite pair (i, -i) with weight w_m and per rest velocity,
//   post_i  = omega w_m rho + a1 f_i + a2 f_-i,  a1,2 = ((1 - omega) +- (1 - omega^j)) / 2
//   post_0  = omega w_0 rho + (1 - omega) f_0
// (15 double operations per D2Q5 node, 9 per D1Q3 node), then push-streaming to
// x + v_i.  No moment matrix appears; the oracle uses the matrix.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ilg_internal.h"

namespace {

constexpr int kLbThreads = 256;
constexpr uint32_t kLbMaxModes = 256;
constexpr uint32_t kLbRowChunk = 64;   // rows per partial column sum
constexpr uint32_t kLbChunk = 4096;    // entries per partial of a projection

struct LbCoef {
  double cr;   // omega w_0
  double cm;   // omega w_m (moving, D2Q9: axis)
  double cd;   // D2Q9: omega w_diagonal
  double l2;   // 1 - omega
  double a1;   // ((1 - omega) + (1 - omega^j)) / 2
  double a2;   // ((1 - omega) - (1 - omega^j)) / 2
};

// One step, one node per thread: blocks stride over rows (blockIdx.y) and over
// x within a row (blockIdx.x); load the Q planes, relax, push.
template <int Q>
__global__ void __launch_bounds__(kLbThreads) lb_step_kernel(LbCoef k, const double* __restrict__ in,
                                                            double* __restrict__ out, uint32_t Lx, uint32_t Ly) {
  const size_t plane = size_t(Lx) * Ly;
  for (uint32_t y = blockIdx.y; y < Ly; y += gridDim.y) {
    const size_t row = size_t(y) * Lx;
    const uint32_t yp = y + 1 == Ly ? 0 : y + 1;
    const uint32_t ym = y == 0 ? Ly - 1 : y - 1;
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < Lx; x += gridDim.x * blockDim.x) {
      const size_t node = row + x;
      double f[Q];
#pragma unroll
      for (int i = 0; i < Q; ++i) f[i] = in[i * plane + node];
      double rho = f[0] + f[1] + f[2];
      if constexpr (Q >= 5) rho = rho + f[3] + f[4];
      if constexpr (Q == 9) rho = rho + f[5] + f[6] + f[7] + f[8];
      const double c = k.cm * rho;
      const double p0 = fma(k.l2, f[0], k.cr * rho);
      const double p1 = fma(k.a1, f[1], fma(k.a2, f[2], c));
      const double p2 = fma(k.a1, f[2], fma(k.a2, f[1], c));
      const uint32_t xp = x + 1 == Lx ? 0 : x + 1;
      const uint32_t xm = x == 0 ? Lx - 1 : x - 1;
      out[node] = p0;
      out[plane + row + xp] = p1;
      out[2 * plane + row + xm] = p2;
      if constexpr (Q >= 5) {
        const double p3 = fma(k.a1, f[3], fma(k.a2, f[4], c));
        const double p4 = fma(k.a1, f[4], fma(k.a2, f[3], c));
        out[3 * plane + size_t(yp) * Lx + x] = p3;
        out[4 * plane + size_t(ym) * Lx + x] = p4;
      }
      if constexpr (Q == 9) {
        // diagonal pairs (+1,+1)/(-1,-1) and (+1,-1)/(-1,+1)
        const double cdr = k.cd * rho;
        const double p5 = fma(k.a1, f[5], fma(k.a2, f[6], cdr));
        const double p6 = fma(k.a1, f[6], fma(k.a2, f[5], cdr));
        const double p7 = fma(k.a1, f[7], fma(k.a2, f[8], cdr));
        const double p8 = fma(k.a1, f[8], fma(k.a2, f[7], cdr));
        out[5 * plane + size_t(yp) * Lx + xp] = p5;
        out[6 * plane + size_t(ym) * Lx + xm] = p6;
        out[7 * plane + size_t(ym) * Lx + xp] = p7;
        out[8 * plane + size_t(yp) * Lx + xm] = p8;
      }
    }
  }
}

// f_i(x, y) = lambda[cls_i * period + r], r the phase residue of the node.
template <int Q>
__global__ void __launch_bounds__(kLbThreads) lb_init_kernel(const double* __restrict__ lam, uint32_t period,
                                                            int axis, uint32_t mode, int weighted,
                                                            double* __restrict__ out, uint32_t Lx, uint32_t Ly) {
  const size_t plane = size_t(Lx) * Ly;
  for (size_t node = size_t(blockIdx.x) * blockDim.x + threadIdx.x; node < plane;
       node += size_t(gridDim.x) * blockDim.x) {
    const uint32_t y = uint32_t(node / Lx);
    const uint32_t x = uint32_t(node - size_t(y) * Lx);
    uint32_t r = 0;
    if (axis == 1) r = uint32_t((uint64_t(mode) * x) % period);
    else if (axis == 2) r = uint32_t((uint64_t(mode) * y) % period);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const uint32_t cls = !weighted || i == 0 ? 0u : (Q == 9 && i > 4 ? 2u : 1u);
      out[i * plane + node] = lam[cls * period + r];
    }
  }
}

// Partial column sums of rho over a chunk of kLbRowChunk rows (fixed order).
template <int Q>
__global__ void __launch_bounds__(kLbThreads) lb_colpart_kernel(const double* __restrict__ f, uint32_t Lx,
                                                               uint32_t Ly, double* __restrict__ part) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Lx) return;
  const size_t plane = size_t(Lx) * Ly;
  const uint32_t y0 = blockIdx.y * kLbRowChunk;
  const uint32_t y1 = y0 + kLbRowChunk < Ly ? y0 + kLbRowChunk : Ly;
  double s = 0.0;
  for (uint32_t y = y0; y < y1; ++y) {
    const size_t at = size_t(y) * Lx + x;
    double n = f[at];
#pragma unroll
    for (int i = 1; i < Q; ++i) n += f[i * plane + at];
    s += n;
  }
  part[size_t(blockIdx.y) * Lx + x] = s;
}

__global__ void lb_colsum_kernel(const double* __restrict__ part, uint32_t Lx, uint32_t chunks,
                                 double* __restrict__ col) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Lx) return;
  double s = 0.0;
  for (uint32_t g = 0; g < chunks; ++g) s += part[size_t(g) * Lx + x];
  col[x] = s;
}

// Row sums of rho: one block per row, strided accumulation, fixed tree.
template <int Q>
__global__ void __launch_bounds__(kLbThreads) lb_rowsum_kernel(const double* __restrict__ f, uint32_t Lx,
                                                              uint32_t Ly, double* __restrict__ row) {
  __shared__ double red[kLbThreads];
  const size_t plane = size_t(Lx) * Ly;
  for (uint32_t y = blockIdx.x; y < Ly; y += gridDim.x) {
    double s = 0.0;
    for (uint32_t x = threadIdx.x; x < Lx; x += blockDim.x) {
      const size_t at = size_t(y) * Lx + x;
      double n = f[at];
#pragma unroll
      for (int i = 1; i < Q; ++i) n += f[i * plane + at];
      s += n;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = kLbThreads / 2; h > 0; h >>= 1) {
      if (int(threadIdx.x) < h) red[threadIdx.x] += red[threadIdx.x + h];
      __syncthreads();
    }
    if (threadIdx.x == 0) row[y] = red[0];
    __syncthreads();
  }
}

// Compensated accumulator: value s plus error term e (Knuth's two-sum; exact
// product errors through fma).  Round-to-nearest intrinsics keep the compiler from
// contracting the error-free transformations.
struct Acc {
  double s = 0.0, e = 0.0;
  __device__ void add(double v) {
    const double t = __dadd_rn(s, v);
    const double bp = __dsub_rn(t, s);
    e = __dadd_rn(e, __dadd_rn(__dsub_rn(s, __dsub_rn(t, bp)), __dsub_rn(v, bp)));
    s = t;
  }
  __device__ void add_product(double a, double b) {
    const double p = __dmul_rn(a, b);
    add(p);
    e = __dadd_rn(e, fma(a, b, -p));
  }
  __device__ void merge(const Acc& o) {
    add(o.s);
    e = __dadd_rn(e, o.e);
  }
};

// Fixed-order block reduction of the threads' accumulators (the same tree for
// every launch shape with kLbThreads threads).
__device__ Acc block_acc(Acc a, double* ss, double* se) {
  ss[threadIdx.x] = a.s;
  se[threadIdx.x] = a.e;
  __syncthreads();
  for (int h = kLbThreads / 2; h > 0; h >>= 1) {
    if (int(threadIdx.x) < h) {
      Acc l{ss[threadIdx.x], se[threadIdx.x]};
      l.merge(Acc{ss[threadIdx.x + h], se[threadIdx.x + h]});
      ss[threadIdx.x] = l.s;
      se[threadIdx.x] = l.e;
    }
    __syncthreads();
  }
  const Acc r{ss[0], se[0]};
  __syncthreads();
  return r;
}

// Partial sums over chunks of kLbChunk consecutive entries; part[c] = (s, e).
__global__ void __launch_bounds__(kLbThreads) lb_mass_partial_kernel(const double* __restrict__ col, uint32_t Lx,
                                                                    double2* __restrict__ part) {
  __shared__ double ss[kLbThreads], se[kLbThreads];
  const uint32_t x0 = blockIdx.x * kLbChunk;
  const uint32_t x1 = x0 + kLbChunk < Lx ? x0 + kLbChunk : Lx;
  Acc a;
  for (uint32_t x = x0 + threadIdx.x; x < x1; x += kLbThreads) a.add(col[x]);
  const Acc r = block_acc(a, ss, se);
  if (threadIdx.x == 0) part[blockIdx.x] = make_double2(r.s, r.e);
}

// Block (c, j): chunk c of mode j; part[(2j) P + c] = re, part[(2j+1) P + c] = im.
// The mean M / L comes from out[0] (the mass, already combined).
__global__ void __launch_bounds__(kLbThreads) lb_mode_partial_kernel(const double* __restrict__ col,
                                                                    const double* __restrict__ row, uint32_t Lx,
                                                                    uint32_t Ly, const int32_t* __restrict__ modes,
                                                                    const double* __restrict__ out,
                                                                    double2* __restrict__ part) {
  __shared__ double ss[kLbThreads], se[kLbThreads];
  const uint32_t j = blockIdx.y, P = gridDim.x;
  const int32_t mx = modes[2 * j], my = modes[2 * j + 1];
  const bool along_x = mx != 0;
  const uint32_t L = along_x ? Lx : Ly;
  const double* C = along_x ? col : row;
  const int64_t mr = along_x ? mx : my;
  const uint64_t mode = uint64_t(((mr % int64_t(L)) + int64_t(L)) % int64_t(L));
  const double mean = out[0] / double(L);
  const uint32_t x0 = blockIdx.x * kLbChunk;
  const uint32_t x1 = x0 + kLbChunk < L ? x0 + kLbChunk : L;
  Acc re, im;
  for (uint32_t x = x0 + threadIdx.x; x < x1; x += kLbThreads) {
    const uint64_t r = (mode * x) % L;
    double sn, cs;
    sincospi(2.0 * double(r) / double(L), &sn, &cs);
    const double d = C[x] - mean;
    re.add_product(cs, d);
    im.add_product(sn, d);
  }
  const Acc a = block_acc(re, ss, se);
  const Acc b = block_acc(im, ss, se);
  if (threadIdx.x == 0) {
    part[size_t(2 * j) * P + blockIdx.x] = make_double2(a.s, a.e);
    part[size_t(2 * j + 1) * P + blockIdx.x] = make_double2(b.s, b.e);
  }
}

// Block q combines part[q P .. q P + P) in a fixed order into out[first + q].
__global__ void __launch_bounds__(kLbThreads) lb_combine_kernel(const double2* __restrict__ part, uint32_t P,
                                                               double* __restrict__ out, uint32_t first) {
  __shared__ double ss[kLbThreads], se[kLbThreads];
  Acc a;
  for (uint32_t c = threadIdx.x; c < P; c += kLbThreads) {
    const double2 v = part[size_t(blockIdx.x) * P + c];
    a.merge(Acc{v.x, v.y});
  }
  const Acc r = block_acc(a, ss, se);
  if (threadIdx.x == 0) out[first + blockIdx.x] = r.s + r.e;
}

}  // namespace

struct ilg_lb {
  ilg_lb_params p{};
  int Q = 3;
  uint32_t Ly = 1;
  size_t nodes = 0;
  cudaStream_t stream = nullptr;
  int sms = 1;
  double* f[2] = {nullptr, nullptr};
  int cur = 0;
  uint64_t t = 0;
  bool has_state = false;
  LbCoef coef{};
  uint32_t chunks = 1;
  double* d_part = nullptr;   // chunks x Lx partial column sums
  double* d_col = nullptr;    // Lx
  double* d_row = nullptr;    // Ly
  double* d_out = nullptr;    // 1 + 2 kLbMaxModes
  double2* d_red = nullptr;   // projection partials, 2 kLbMaxModes x chunks
  int32_t* d_modes = nullptr; // 2 kLbMaxModes
  std::string err;
};

namespace {

ilg_status lb_fail(ilg_lb* b, ilg_status s, const std::string& msg) {
  if (b) b->err = msg;
  else ilg::set_context_free_error(msg);
  return s;
}

ilg_status lb_cuda_fail(ilg_lb* b, cudaError_t e, const char* what) {
  return lb_fail(b, e == cudaErrorMemoryAllocation ? ILG_E_OOM : ILG_E_CUDA,
                 std::string(what) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(b, call, what)                             \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return lb_cuda_fail(b, e_, what); \
  } while (0)

// The gas's parameters that define the same lattice and initial means.
ilg_params as_gas(const ilg_lb_params& p) {
  ilg_params g{};
  g.lattice = p.lattice;
  g.Lx = p.Lx;
  g.Ly = p.Ly;
  g.mode_mx = p.mode_mx;
  g.mode_my = p.mode_my;
  g.init_weighted = p.init_weighted;
  g.n0 = p.n0;
  g.amp = p.amp;
  g.omega_eff = 1.0;
  g.theta = p.theta;
  return g;
}

int lb_grid(const ilg_lb* b) {
  const size_t blocks = (b->nodes + kLbThreads - 1) / kLbThreads;
  const size_t cap = size_t(b->sms) * (2048 / kLbThreads);
  return int(blocks < cap ? blocks : cap);
}

// step grid: x blocks cover a row (up to the resident total), y blocks share rows
dim3 lb_step_grid(const ilg_lb* b) {
  const uint32_t cap = uint32_t(b->sms) * (2048 / kLbThreads);
  uint32_t gx = (b->p.Lx + kLbThreads - 1) / kLbThreads;
  if (gx > cap) gx = cap;
  uint32_t gy = cap / gx;
  if (gy < 1) gy = 1;
  if (gy > b->Ly) gy = b->Ly;
  return dim3(gx, gy);
}

}  // namespace

extern "C" {

ilg_status ilg_lb_create(const ilg_lb_params* params, void* stream, ilg_lb** out) {
  if (!out) return lb_fail(nullptr, ILG_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!params) return lb_fail(nullptr, ILG_E_INVALID, "params is NULL");
  const ilg_lb_params& p = *params;
  const std::string why = ilg::validate_params(as_gas(p));
  if (!why.empty()) return lb_fail(nullptr, ILG_E_INVALID, why);
  if (!(p.omega_j >= 0.0 && p.omega_j <= 2.0)) return lb_fail(nullptr, ILG_E_INVALID, "omega_j must lie in [0, 2]");
  if (!(p.omega >= 0.0 && p.omega <= 2.0)) return lb_fail(nullptr, ILG_E_INVALID, "omega must lie in [0, 2]");
  ilg_lb* b = new ilg_lb();
  b->p = p;
  b->Q = p.lattice == ILG_D1Q3 ? 3 : (p.lattice == ILG_D2Q5 ? 5 : 9);
  b->Ly = p.lattice == ILG_D1Q3 ? 1 : p.Ly;
  b->p.Ly = b->Ly;
  b->nodes = size_t(p.Lx) * b->Ly;
  b->stream = static_cast<cudaStream_t>(stream);
  double w[9];
  ilg::weights(p.lattice, p.theta, w);
  const double l2 = 1.0 - p.omega, lj = 1.0 - p.omega_j;
  b->coef = LbCoef{p.omega * w[0], p.omega * w[1], b->Q == 9 ? p.omega * w[5] : 0.0, l2, 0.5 * (l2 + lj),
                   0.5 * (l2 - lj)};
  b->chunks = (b->Ly + kLbRowChunk - 1) / kLbRowChunk;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  const size_t bytes = sizeof(double) * b->Q * b->nodes;
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->f[0], bytes);
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->f[1], bytes);
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->d_part, sizeof(double) * b->chunks * p.Lx);
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->d_col, sizeof(double) * p.Lx);
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->d_row, sizeof(double) * b->Ly);
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->d_out, sizeof(double) * (1 + 2 * kLbMaxModes));
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->d_modes, sizeof(int32_t) * 2 * kLbMaxModes);
  const size_t maxL = p.Lx > b->Ly ? p.Lx : b->Ly;
  if (e == cudaSuccess) e = ilg::dev_alloc(&b->d_red, sizeof(double2) * 2 * kLbMaxModes * ((maxL + kLbChunk - 1) / kLbChunk));
  if (e != cudaSuccess) {
    ilg_lb_destroy(b);
    return lb_cuda_fail(nullptr, e, "ilg_lb_create");
  }
  *out = b;
  return ILG_OK;
}

ilg_status ilg_lb_destroy(ilg_lb* b) {
  if (!b) return ILG_E_INVALID;
  if (b->f[0] || b->f[1]) cudaStreamSynchronize(b->stream);
  cudaFree(b->f[0]);
  cudaFree(b->f[1]);
  cudaFree(b->d_part);
  cudaFree(b->d_col);
  cudaFree(b->d_row);
  cudaFree(b->d_out);
  cudaFree(b->d_modes);
  cudaFree(b->d_red);
  delete b;
  return ILG_OK;
}

const char* ilg_lb_last_error(const ilg_lb* b) { return b ? b->err.c_str() : ilg_last_error(nullptr); }

// Sec. IV, Eq. omegaj: with the flip (omega_eff > 1) the collision fraction is
// omega* = 2 - omega_eff; the current then relaxes with omega^j = 2 - omega* and the
// even moments with omega*.  Without the flip every non-conserved moment relaxes with
// omega_eff.
ilg_status ilg_lb_rates(double omega_eff, double* omega_j, double* omega) {
  if (!omega_j || !omega || !(omega_eff > 0.0 && omega_eff <= 2.0)) {
    ilg::set_context_free_error("ilg_lb_rates: omega_eff must lie in (0, 2] and the outputs be non-NULL");
    return ILG_E_INVALID;
  }
  *omega_j = omega_eff;
  *omega = omega_eff > 1.0 ? 2.0 - omega_eff : omega_eff;
  return ILG_OK;
}

ilg_status ilg_lb_init(ilg_lb* b) {
  if (!b) return ILG_E_INVALID;
  const ilg_params g = as_gas(b->p);
  const uint32_t period = ilg::initial_period(g);
  const int classes = b->p.init_weighted ? (b->Q == 9 ? 3 : 2) : 1;
  std::vector<double> lam(size_t(classes) * period);
  for (int c = 0; c < classes; ++c)
    for (uint32_t r = 0; r < period; ++r) {
      const double v = ilg::initial_mean(g, b->Q, c, r, period);
      if (!(v >= 0.0) || v > ilg::kMaxMean)
        return lb_fail(b, ILG_E_INVALID, "initial mean " + std::to_string(v) + " outside [0, 700]");
      lam[size_t(c) * period + r] = v;
    }
  int axis = 0;
  uint32_t mode = 0;
  if (period > 1) {
    const bool along_x = b->p.mode_mx != 0;
    const int64_t L = period, m = along_x ? b->p.mode_mx : b->p.mode_my;
    axis = along_x ? 1 : 2;
    mode = uint32_t(((m % L) + L) % L);
  }
  double* d_lam = nullptr;
  LB_CUDA(b, ilg::dev_alloc(&d_lam, sizeof(double) * lam.size()), "cudaMalloc");
  cudaError_t e = cudaMemcpyAsync(d_lam, lam.data(), sizeof(double) * lam.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) {
    if (b->Q == 3)
      lb_init_kernel<3><<<lb_grid(b), kLbThreads, 0, b->stream>>>(d_lam, period, axis, mode, b->p.init_weighted,
                                                                  b->f[b->cur], b->p.Lx, b->Ly);
    else if (b->Q == 5)
      lb_init_kernel<5><<<lb_grid(b), kLbThreads, 0, b->stream>>>(d_lam, period, axis, mode, b->p.init_weighted,
                                                                  b->f[b->cur], b->p.Lx, b->Ly);
    else
      lb_init_kernel<9><<<lb_grid(b), kLbThreads, 0, b->stream>>>(d_lam, period, axis, mode, b->p.init_weighted,
                                                                  b->f[b->cur], b->p.Lx, b->Ly);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(d_lam);
  if (e != cudaSuccess) return lb_cuda_fail(b, e, "lattice Boltzmann init");
  b->t = 0;
  b->has_state = true;
  return ILG_OK;
}

ilg_status ilg_lb_set_state(ilg_lb* b, const double* host, size_t n, uint64_t t) {
  if (!b) return ILG_E_INVALID;
  if (!host || n != size_t(b->Q) * b->nodes) return lb_fail(b, ILG_E_INVALID, "state must hold Q*Lx*Ly doubles");
  LB_CUDA(b, cudaMemcpyAsync(b->f[b->cur], host, sizeof(double) * n, cudaMemcpyHostToDevice, b->stream), "copy in");
  LB_CUDA(b, cudaStreamSynchronize(b->stream), "copy in");
  b->t = t;
  b->has_state = true;
  return ILG_OK;
}

ilg_status ilg_lb_get_state(ilg_lb* b, double* host, size_t n, uint64_t* t) {
  if (!b) return ILG_E_INVALID;
  if (!b->has_state) return lb_fail(b, ILG_E_STATE, "no state: call ilg_lb_init or ilg_lb_set_state first");
  if (!host || n != size_t(b->Q) * b->nodes) return lb_fail(b, ILG_E_INVALID, "state must hold Q*Lx*Ly doubles");
  LB_CUDA(b, cudaMemcpyAsync(host, b->f[b->cur], sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream), "copy out");
  LB_CUDA(b, cudaStreamSynchronize(b->stream), "copy out");
  if (t) *t = b->t;
  return ILG_OK;
}

ilg_status ilg_lb_step(ilg_lb* b, uint32_t T) {
  if (!b) return ILG_E_INVALID;
  if (!b->has_state) return lb_fail(b, ILG_E_STATE, "no state: call ilg_lb_init or ilg_lb_set_state first");
  const dim3 grid = lb_step_grid(b);
  for (uint32_t k = 0; k < T; ++k) {
    if (b->Q == 3)
      lb_step_kernel<3><<<grid, kLbThreads, 0, b->stream>>>(b->coef, b->f[b->cur], b->f[b->cur ^ 1], b->p.Lx, b->Ly);
    else if (b->Q == 5)
      lb_step_kernel<5><<<grid, kLbThreads, 0, b->stream>>>(b->coef, b->f[b->cur], b->f[b->cur ^ 1], b->p.Lx, b->Ly);
    else
      lb_step_kernel<9><<<grid, kLbThreads, 0, b->stream>>>(b->coef, b->f[b->cur], b->f[b->cur ^ 1], b->p.Lx, b->Ly);
    LB_CUDA(b, cudaGetLastError(), "lattice Boltzmann step");
    b->cur ^= 1;
    b->t += 1;
  }
  return ILG_OK;
}

ilg_status ilg_lb_observables(ilg_lb* b, const int32_t* modes, uint32_t nmodes, uint64_t* t, double* mass,
                              double* re, double* im, double* amp) {
  if (!b) return ILG_E_INVALID;
  if (!b->has_state) return lb_fail(b, ILG_E_STATE, "no state: call ilg_lb_init or ilg_lb_set_state first");
  if (nmodes > kLbMaxModes) return lb_fail(b, ILG_E_INVALID, "at most 256 modes");
  if (nmodes && !modes) return lb_fail(b, ILG_E_INVALID, "modes is NULL");
  bool any_y = false;
  for (uint32_t j = 0; j < nmodes; ++j) {
    const int32_t mx = modes[2 * j], my = modes[2 * j + 1];
    if ((mx == 0) == (my == 0)) return lb_fail(b, ILG_E_INVALID, "each mode must be an axis mode");
    if (b->p.lattice == ILG_D1Q3 && my != 0) return lb_fail(b, ILG_E_INVALID, "D1Q3 has no y mode");
    any_y |= my != 0;
  }
  const uint32_t Lx = b->p.Lx, Ly = b->Ly;
  const double* f = b->f[b->cur];
  const dim3 pg((Lx + kLbThreads - 1) / kLbThreads, b->chunks);
  if (b->Q == 3) lb_colpart_kernel<3><<<pg, kLbThreads, 0, b->stream>>>(f, Lx, Ly, b->d_part);
  else if (b->Q == 5) lb_colpart_kernel<5><<<pg, kLbThreads, 0, b->stream>>>(f, Lx, Ly, b->d_part);
  else lb_colpart_kernel<9><<<pg, kLbThreads, 0, b->stream>>>(f, Lx, Ly, b->d_part);
  LB_CUDA(b, cudaGetLastError(), "column sums");
  lb_colsum_kernel<<<pg.x, kLbThreads, 0, b->stream>>>(b->d_part, Lx, b->chunks, b->d_col);
  LB_CUDA(b, cudaGetLastError(), "column sums");
  if (any_y) {
    const int rg = int(Ly < uint32_t(b->sms) * 8 ? Ly : uint32_t(b->sms) * 8);
    if (b->Q == 3) lb_rowsum_kernel<3><<<rg, kLbThreads, 0, b->stream>>>(f, Lx, Ly, b->d_row);
    else if (b->Q == 5) lb_rowsum_kernel<5><<<rg, kLbThreads, 0, b->stream>>>(f, Lx, Ly, b->d_row);
    else lb_rowsum_kernel<9><<<rg, kLbThreads, 0, b->stream>>>(f, Lx, Ly, b->d_row);
    LB_CUDA(b, cudaGetLastError(), "row sums");
  }
  if (nmodes)
    LB_CUDA(b, cudaMemcpyAsync(b->d_modes, modes, sizeof(int32_t) * 2 * nmodes, cudaMemcpyHostToDevice, b->stream),
            "copy modes");
  const uint32_t Pm = (Lx + kLbChunk - 1) / kLbChunk;
  lb_mass_partial_kernel<<<Pm, kLbThreads, 0, b->stream>>>(b->d_col, Lx, b->d_red);
  LB_CUDA(b, cudaGetLastError(), "mass");
  lb_combine_kernel<<<1, kLbThreads, 0, b->stream>>>(b->d_red, Pm, b->d_out, 0);
  LB_CUDA(b, cudaGetLastError(), "mass");
  if (nmodes) {
    const uint32_t maxL = Lx > Ly ? Lx : Ly;
    const uint32_t P = (maxL + kLbChunk - 1) / kLbChunk;
    lb_mode_partial_kernel<<<dim3(P, nmodes), kLbThreads, 0, b->stream>>>(b->d_col, b->d_row, Lx, Ly, b->d_modes,
                                                                          b->d_out, b->d_red);
    LB_CUDA(b, cudaGetLastError(), "projection");
    lb_combine_kernel<<<2 * nmodes, kLbThreads, 0, b->stream>>>(b->d_red, P, b->d_out, 1);
    LB_CUDA(b, cudaGetLastError(), "projection");
  }
  std::vector<double> h(1 + 2 * size_t(nmodes));
  LB_CUDA(b, cudaMemcpyAsync(h.data(), b->d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, b->stream),
          "copy observables");
  LB_CUDA(b, cudaStreamSynchronize(b->stream), "observables");
  if (t) *t = b->t;
  if (mass) *mass = h[0];
  const double half = double(Lx) * double(Ly) / 2.0;
  for (uint32_t j = 0; j < nmodes; ++j) {
    if (re) re[j] = h[1 + 2 * j];
    if (im) im[j] = h[2 + 2 * j];
    if (amp) amp[j] = h[2 + 2 * j] / half;
  }
  return ILG_OK;
}

}  // extern "C"
