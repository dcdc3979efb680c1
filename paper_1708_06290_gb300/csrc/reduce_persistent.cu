// Controller-Hessenberg reduction (Algorithm 1, Sec. 2) as ONE persistent
// cooperative kernel.  Every reflector H = I - tau v v^T is applied two-sided
// in four phases separated by a grid barrier:
//   1. block 0 generates the reflector of the current column (and, while B is
//      being triangularised, applies it to the remaining columns of B);
//   2. all blocks: column dots u = A^T v and row dots w = A v (and C v) over
//      shared-memory-staged tiles, partial sums per tile;
//   3. all blocks: reduce the partial sums (u, w, s = u^T v);
//   4. all blocks: A <- A - tau v u^T - tau w' v^T with w' = w - tau s v
//      (= H A H), C <- C - tau w_C v^T.
// The barrier is the library's own: it spins with a bounded iteration count
// and, if the count runs out, raises an error flag so every block returns and
// the host reports SSV_ETIMEOUT.  The cooperative launch guarantees that all
// blocks are resident, so in normal operation every wait ends.
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {

namespace {

constexpr int kT = 256;          // threads per block
constexpr int kPR = 64;          // tile rows
constexpr int kPC = 128;         // tile columns
constexpr int kPLD = kPR + 1;    // padded shared-memory column stride (odd)
constexpr unsigned long long kBarrierSpins = 1ull << 28;  // ~10 s of 32 ns naps

struct RedArgs {
  double* H;
  double* R;
  double* Ct;
  double* tauA;
  double* tauB;
  int n, m, p, ldct, kb, ka;
  double* upart;   // nrt_max x n
  double* wpart;   // nct_max x (n + p)
  double* spart;   // nrt_max x nct_max
  double* u;       // n
  double* w;       // n + p
  double* s;       // 1
  unsigned* bar;   // [0] arrivals, [1] generation
  int* err;        // 1 after a barrier timed out
};

constexpr size_t kSmemDoubles = (size_t)kPC * kPLD + kPC + kPR + 4 * kPR + 8;

// Data written by other blocks in an earlier phase is read with __ldcg (L2,
// not the SM's L1, which is not coherent across SMs).
__device__ __forceinline__ double vrow(int i, int r0, int n, const double* __restrict__ v) {
  return (i >= r0 && i < n) ? (i == r0 ? 1.0 : __ldcg(v + (i - r0))) : 0.0;
}

// Grid-wide barrier with a bounded wait.  Returns false once any block has
// given up (then every block leaves the kernel).
__device__ bool grid_barrier(unsigned* bar, int* err, unsigned long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*gen == g) {
        if (*(volatile int*)err != 0) break;
        if (++spins > limit) {
          atomicExch(err, 1);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    s_ok = (*(volatile int*)err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Householder vector of x (len entries) by one block: beta = -sign(alpha)||x||,
// tau = (beta - alpha)/beta, x(1:) scaled by 1/(alpha - beta), x(0) = beta.
__device__ void house_block(double* __restrict__ x, int len, double* __restrict__ tau_out,
                            double* red) {
  double ss = 0.0;
  for (int i = 1 + threadIdx.x; i < len; i += kT) {
    const double xi = __ldcg(x + i);
    ss = fma(xi, xi, ss);
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int k = 0; k < kT / 32; ++k) v += red[k];
    const double alpha = __ldcg(x);
    double tau = 0.0, scal = 0.0;
    if (len > 1 && v != 0.0) {
      const double nrm = sqrt(fma(alpha, alpha, v));
      const double beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
      x[0] = beta;
    }
    *tau_out = tau;
    red[0] = scal;
  }
  __syncthreads();
  const double scal = red[0];
  if (scal != 0.0)
    for (int i = 1 + threadIdx.x; i < len; i += kT) x[i] = __ldcg(x + i) * scal;
  __syncthreads();
}

// Left application of the B-reflector to columns c0..c1-1 of R (rows r0..),
// one warp per column (block 0 only; at most m - 1 columns).
__device__ void left_R(double* __restrict__ R, int n, int r0, int len, int c0, int c1,
                       const double* __restrict__ v, double tau) {
  if (tau == 0.0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = c0 + warp; c < c1; c += kT / 32) {
    double* col = R + (size_t)c * n + r0;
    double d = 0.0;
    for (int i = lane; i < len; i += 32) d = fma(i == 0 ? 1.0 : v[i], __ldcg(col + i), d);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const double wv = tau * d;
    for (int i = lane; i < len; i += 32) col[i] = fma(-(i == 0 ? 1.0 : v[i]), wv, __ldcg(col + i));
  }
}

// Phase 2 on one tile: stage it in shared memory, row dots and column dots.
__device__ void dots_tile(const RedArgs& a, int ct, int rt, int nct, int r0, int cl,
                          const double* __restrict__ v, double* fsm) {
  const int n = a.n, np = a.n + a.p;
  double* tile = fsm;
  double* vc_s = tile + kPC * kPLD;
  double* vr_s = vc_s + kPC;
  double* wq = vr_s + kPR;
  double* red = wq + 4 * kPR;
  const int tid = threadIdx.x;
  const int c0 = cl + ct * kPC, i0 = rt * kPR;
  __syncthreads();
  if (tid < kPC) vc_s[tid] = (c0 + tid < n) ? vrow(c0 + tid, r0, n, v) : 0.0;
  if (tid < kPR) vr_s[tid] = vrow(i0 + tid, r0, n, v);
#pragma unroll 8
  for (int k = 0; k < (kPR * kPC) / kT; ++k) {
    const int idx = k * kT + tid;
    const int r = idx % kPR, c = idx / kPR;
    const int i = i0 + r, cg = c0 + c;
    double x = 0.0;
    if (cg < n) {
      if (i < n) x = __ldcg(a.H + i + (size_t)cg * n);
      else if (i < np) x = __ldcg(a.Ct + (i - n) + (size_t)cg * a.ldct);
    }
    tile[c * kPLD + r] = x;
  }
  __syncthreads();
  {
    const int r = tid % kPR, qtr = tid / kPR;
    double acc = 0.0;
#pragma unroll 8
    for (int c = qtr * 32; c < qtr * 32 + 32; ++c) acc = fma(tile[c * kPLD + r], vc_s[c], acc);
    wq[qtr * kPR + r] = acc;
  }
  double u = 0.0;
  if (tid < kPC) {
#pragma unroll 8
    for (int r = 0; r < kPR; ++r) u = fma(vr_s[r], tile[tid * kPLD + r], u);
  }
  __syncthreads();
  if (tid < kPR) {
    const int ii = i0 + tid;
    if (ii < np)
      a.wpart[(size_t)ct * np + ii] = wq[tid] + wq[kPR + tid] + wq[2 * kPR + tid] + wq[3 * kPR + tid];
  }
  double sp = 0.0;
  if (tid < kPC) {
    if (c0 + tid < n) a.upart[(size_t)rt * n + c0 + tid] = u;
    sp = u * vc_s[tid];
  }
  for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
  if ((tid & 31) == 0) red[tid >> 5] = sp;
  __syncthreads();
  if (tid == 0) a.spart[(size_t)rt * nct + ct] = red[0] + red[1] + red[2] + red[3];
}

// Phase 4 on one tile: A -= tau v u^T (rows >= r0, columns >= cl) + tau w' v^T.
__device__ void update_tile(const RedArgs& a, int ct, int rt, int r0, int cl,
                            const double* __restrict__ v, double tau, double* fsm) {
  const int n = a.n, np = a.n + a.p;
  double* vc_s = fsm;
  double* tu_s = vc_s + kPC;
  const int tid = threadIdx.x;
  const int c0 = cl + ct * kPC;
  __syncthreads();
  if (tid < kPC) {
    const int c = c0 + tid;
    vc_s[tid] = (c < n) ? vrow(c, r0, n, v) : 0.0;
    tu_s[tid] = (c < n) ? tau * __ldcg(a.u + c) : 0.0;
  }
  __syncthreads();
  const int r = tid % kPR, qtr = tid / kPR;
  const int i = rt * kPR + r;
  if (i >= np) return;
  const double vi = vrow(i, r0, n, v);
  const double twp = tau * (__ldcg(a.w + i) - tau * __ldcg(a.s) * vi);
  const double lvi = (i >= r0 && i < n) ? vi : 0.0;
  const int cb = c0 + qtr * 32;
  const int cnt = min(32, n - cb);
  if (cnt <= 0) return;
  double* base = i < n ? a.H + i : a.Ct + (i - n);
  const size_t ld = i < n ? (size_t)n : (size_t)a.ldct;
  double x[32];
#pragma unroll
  for (int k = 0; k < 32; ++k)
    if (k < cnt) x[k] = __ldcg(base + (size_t)(cb + k) * ld);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < cnt) {
      const int cc = qtr * 32 + k;
      const double t = fma(-lvi, tu_s[cc], x[k]);
      base[(size_t)(cb + k) * ld] = fma(-twp, vc_s[cc], t);
    }
  }
}

__global__ void __launch_bounds__(kT) reduce_persistent_kernel(RedArgs a) {
  extern __shared__ double fsm[];
  __shared__ double red[kT / 32];
  const int n = a.n, m = a.m, np = a.n + a.p;
  const int nrefl = a.kb + a.ka;
  for (int t = 0; t < nrefl; ++t) {
    const bool bphase = t < a.kb;
    const int idx = bphase ? t : t - a.kb;
    const int r0 = bphase ? idx : idx + m;
    const int cl = bphase ? 0 : idx + 1;
    const int len = n - r0;
    double* x = bphase ? a.R + idx + (size_t)idx * n : a.H + r0 + (size_t)idx * n;
    double* tau_p = bphase ? a.tauB + idx : a.tauA + idx;
    if (len <= 1) continue;  // uniform: no reflector to apply
    // phase 1
    if (blockIdx.x == 0) {
      house_block(x, len, tau_p, red);
      if (bphase) left_R(a.R, n, r0, len, idx + 1, m, x, *tau_p);
    }
    if (!grid_barrier(a.bar, a.err, kBarrierSpins)) return;
    const double tau = *(volatile double*)tau_p;
    if (tau == 0.0) continue;  // uniform after the barrier
    const int nrt = (np + kPR - 1) / kPR;
    const int nct = (n - cl + kPC - 1) / kPC;
    // phase 2
    for (int tile = blockIdx.x; tile < nrt * nct; tile += gridDim.x)
      dots_tile(a, tile % nct, tile / nct, nct, r0, cl, x, fsm);
    if (!grid_barrier(a.bar, a.err, kBarrierSpins)) return;
    // phase 3
    for (int e = blockIdx.x * kT + threadIdx.x; e < np; e += gridDim.x * kT) {
      if (e >= cl && e < n) {
        double s = 0.0;
        for (int r = 0; r < nrt; ++r) s += __ldcg(a.upart + (size_t)r * n + e);
        a.u[e] = s;
      }
      double s2 = 0.0;
      for (int c = 0; c < nct; ++c) s2 += __ldcg(a.wpart + (size_t)c * np + e);
      a.w[e] = s2;
    }
    if (blockIdx.x == 0) {
      double s3 = 0.0;
      for (int k = threadIdx.x; k < nrt * nct; k += kT) s3 += __ldcg(a.spart + k);
      for (int o = 16; o > 0; o >>= 1) s3 += __shfl_xor_sync(0xffffffffu, s3, o);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s3;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int k = 0; k < kT / 32; ++k) tot += red[k];
        *a.s = tot;
      }
    }
    if (!grid_barrier(a.bar, a.err, kBarrierSpins)) return;
    // phase 4
    for (int tile = blockIdx.x; tile < nrt * nct; tile += gridDim.x)
      update_tile(a, tile % nct, tile / nct, r0, cl, x, tau, fsm);
    if (!grid_barrier(a.bar, a.err, kBarrierSpins)) return;
  }
}

// Self-test of the bounded barrier: block 0 never arrives, the others must give
// up after `limit` naps and raise the flag.
__global__ void barrier_selftest_kernel(unsigned* bar, int* err, unsigned long long limit) {
  if (blockIdx.x == 0) return;
  grid_barrier(bar, err, limit);
}

}  // namespace

int reduce_persistent(Handle* h, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  const int np = n + p;
  h->kb = std::min(m, n - 1);
  h->ka = std::max(0, n - m - 1);
  const size_t nrt_max = (size_t)(np + kPR - 1) / kPR;
  const size_t nct_max = (size_t)(n + kPC - 1) / kPC;
  const size_t ndbl = nrt_max * n + nct_max * np + nrt_max * nct_max + n + np + 1;
  const size_t bytes = sizeof(double) * ndbl + 4 * sizeof(unsigned) + 16;
  unsigned char* wsp = nullptr;
  SSV_CUDA_TRY(cudaMallocAsync((void**)&wsp, bytes, st));
  RedArgs a;
  a.H = h->H; a.R = h->R; a.Ct = h->Ct; a.tauA = h->tauA; a.tauB = h->tauB;
  a.n = n; a.m = m; a.p = p; a.ldct = p > 0 ? p : 1; a.kb = h->kb; a.ka = h->ka;
  double* d = reinterpret_cast<double*>(wsp);
  a.upart = d;
  a.wpart = a.upart + nrt_max * n;
  a.spart = a.wpart + nct_max * np;
  a.u = a.spart + nrt_max * nct_max;
  a.w = a.u + n;
  a.s = a.w + np;
  a.bar = reinterpret_cast<unsigned*>(d + ndbl);
  a.err = reinterpret_cast<int*>(a.bar + 2);
  int rc = SSV_OK;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), st);
  const size_t smem = sizeof(double) * kSmemDoubles;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reduce_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reduce_persistent_kernel, kT, smem);
  if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) {
    const int grid = num_sms() * std::min(occ, 2);
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)reduce_persistent_kernel, dim3(grid), dim3(kT), args,
                                    smem, st);
    count_launch();
  }
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, a.err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    rc = e == cudaErrorMemoryAllocation ? SSV_ENOMEM : SSV_ECUDA;
  } else if (herr != 0) {
    rc = SSV_ETIMEOUT;
  }
  cudaError_t e2 = cudaFreeAsync(wsp, st);
  if (e2 != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e2);
    rc = SSV_ECUDA;
  }
  return rc;
}

int barrier_selftest(long long limit, cudaStream_t st) {
  unsigned char* wsp = nullptr;
  SSV_CUDA_TRY(cudaMallocAsync((void**)&wsp, 16, st));
  unsigned* bar = reinterpret_cast<unsigned*>(wsp);
  int* err = reinterpret_cast<int*>(bar + 2);
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(wsp, 0, 16, st);
  if (e == cudaSuccess) {
    void* args[] = {&bar, &err, &limit};
    e = cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(4), dim3(kT), args, 0,
                                    st);
    count_launch();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(wsp, st);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return SSV_ECUDA;
  }
  return herr ? SSV_ETIMEOUT : SSV_OK;
}

}  // namespace ssv
