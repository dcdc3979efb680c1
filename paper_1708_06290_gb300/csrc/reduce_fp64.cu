// Controller-Hessenberg reduction in FP64 on the GPU (Algorithm 1, Sec. 2).
//
// Step 1  QR of B with Householder reflectors (one per column of B).
// Step 2  each B-reflector applied to A from both sides and to C from the right.
// Step 3  for column j, a reflector acting on rows j+m .. n-1 annihilates
//         A(j+m+1 : n-1, j); applied from the left to the trailing columns,
//         from the right to all rows of A and to C (Step 4, C <- C Q_A).
//
// The reflector H = I - tau v v^T with v(0) = 1 is generated in the
// annihilated column itself: beta is stored at the top and v(1:) below it,
// as LAPACK stores reflectors, so Q can be applied later (ssv_apply_q).
// The solver reads only the structural part of H (rows <= column + m).
//
// Every kernel is stream-ordered; tau never leaves the device.
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {

namespace {

constexpr int kHouseThreads = 1024;

// x = [alpha; x2] (len entries, contiguous).  Computes beta = -sign(alpha)||x||,
// tau = (beta - alpha)/beta, scales x2 by 1/(alpha - beta), stores beta in x[0].
// tau = 0 (identity) when x2 == 0.
__global__ void __launch_bounds__(kHouseThreads) house_kernel(double* __restrict__ x, int len,
                                                              double* __restrict__ tau_out) {
  __shared__ double red[kHouseThreads / 32];
  __shared__ double s_scal;
  double ss = 0.0;
  for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) ss = fma(x[i], x[i], ss);
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ss;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) {
      double alpha = x[0];
      double tau = 0.0, scal = 0.0;
      if (len > 1 && v != 0.0) {
        double nrm = sqrt(fma(alpha, alpha, v));
        double beta = alpha >= 0.0 ? -nrm : nrm;
        tau = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
        x[0] = beta;
      }
      *tau_out = tau;
      s_scal = scal;
    }
  }
  __syncthreads();
  double scal = s_scal;
  if (scal != 0.0)
    for (int i = 1 + threadIdx.x; i < len; i += blockDim.x) x[i] *= scal;
}

// Left application to columns [c0, c1) of a (ld), rows r0 .. r0+len-1:
// w = v^T a(:, c), a(:, c) -= tau v w.  v(0) = 1, v(1:) = vsrc[1:].
// One warp per column.
__global__ void __launch_bounds__(256) apply_left_kernel(double* __restrict__ a, long long ld,
                                                         int r0, int len, int c0, int c1,
                                                         const double* __restrict__ vsrc,
                                                         const double* __restrict__ tau_p) {
  double tau = *tau_p;
  if (tau == 0.0) return;
  int lane = threadIdx.x & 31;
  int col = c0 + (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (col >= c1) return;
  double* x = a + (size_t)col * ld + r0;
  double dot = 0.0;
  for (int i = lane; i < len; i += 32) {
    double v = i == 0 ? 1.0 : vsrc[i];
    dot = fma(v, x[i], dot);
  }
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  double w = tau * dot;
  for (int i = lane; i < len; i += 32) {
    double v = i == 0 ? 1.0 : vsrc[i];
    x[i] = fma(-v, w, x[i]);
  }
}

// ---------------------------------------------------------------------------
// Two-sided application of one reflector H = I - tau v v^T (v(r0) = 1,
// support rows/columns r0 .. n-1) to A (n x n) and, from the right, to C
// (p x n), in two passes over the matrix:
//   u_c = sum_{i >= r0} v_i A(i, c)       (c >= cl: the left-update columns)
//   w_i = sum_{c >= r0} A(i, c) v_c       (all rows of A, then the rows of C)
//   s   = u^T v
//   A <- A - tau v u^T - tau w' v^T,  w' = w - tau s v   (= H A H),
//   C <- C - tau w_C v^T.
// The left update touches rows >= r0 of columns >= cl only (columns left of
// cl hold stored reflectors there).  Rows of C follow the rows of A as
// "virtual" rows n .. n+p-1.  Partial sums are reduced in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kFR = 64;   // tile rows
constexpr int kFC = 128;  // tile columns
constexpr int kFLD = kFR + 1;  // padded shared-memory column stride (odd: conflict-free)

__device__ __forceinline__ double vrow(int i, int r0, int n, const double* __restrict__ vsrc) {
  return (i >= r0 && i < n) ? (i == r0 ? 1.0 : vsrc[i - r0]) : 0.0;
}

// Pass 1: the tile is staged once in shared memory (coalesced loads); row dots
// w and column dots u are both read from there.
__global__ void __launch_bounds__(256) fused_dots_kernel(
    const double* __restrict__ A, int n, const double* __restrict__ C, int ldc, int p, int r0,
    int cl, const double* __restrict__ vsrc, const double* __restrict__ tau_p,
    double* __restrict__ upart, double* __restrict__ wpart, double* __restrict__ spart) {
  if (*tau_p == 0.0) return;
  extern __shared__ double fsm[];
  double* tile = fsm;                       // kFC columns x kFLD
  double* vc_s = tile + kFC * kFLD;         // kFC
  double* vr_s = vc_s + kFC;                // kFR
  double* wq = vr_s + kFR;                  // 4 x kFR
  double* red = wq + 4 * kFR;               // 8
  const int tid = threadIdx.x;
  const int rt = blockIdx.y, ct = blockIdx.x;
  const int c0 = cl + ct * kFC, i0 = rt * kFR;
  const int np = n + p;
  if (tid < kFC) vc_s[tid] = (c0 + tid < n) ? vrow(c0 + tid, r0, n, vsrc) : 0.0;
  if (tid < kFR) vr_s[tid] = vrow(i0 + tid, r0, n, vsrc);
#pragma unroll 8
  for (int k = 0; k < (kFR * kFC) / 256; ++k) {
    const int idx = k * 256 + tid;
    const int r = idx % kFR, c = idx / kFR;
    const int i = i0 + r, cg = c0 + c;
    double a = 0.0;
    if (cg < n) {
      if (i < n) a = A[i + (size_t)cg * n];
      else if (i < np) a = C[(i - n) + (size_t)cg * ldc];
    }
    tile[c * kFLD + r] = a;
  }
  __syncthreads();
  // row dots: thread (r, quarter) sums 32 columns
  {
    const int r = tid % kFR, qtr = tid / kFR;
    double acc = 0.0;
#pragma unroll 8
    for (int c = qtr * 32; c < qtr * 32 + 32; ++c) acc = fma(tile[c * kFLD + r], vc_s[c], acc);
    wq[qtr * kFR + r] = acc;
  }
  // column dots: threads 0..127, one column each over the 64 rows
  double u = 0.0;
  if (tid < kFC) {
#pragma unroll 8
    for (int r = 0; r < kFR; ++r) u = fma(vr_s[r], tile[tid * kFLD + r], u);
  }
  __syncthreads();
  if (tid < kFR) {
    const int ii = i0 + tid;
    if (ii < np) wpart[(size_t)ct * np + ii] = wq[tid] + wq[kFR + tid] + wq[2 * kFR + tid] + wq[3 * kFR + tid];
  }
  double sp = 0.0;
  if (tid < kFC) {
    if (c0 + tid < n) upart[(size_t)rt * n + c0 + tid] = u;
    sp = u * vc_s[tid];
  }
  for (int o = 16; o > 0; o >>= 1) sp += __shfl_xor_sync(0xffffffffu, sp, o);
  if ((tid & 31) == 0) red[tid >> 5] = sp;
  __syncthreads();
  if (tid == 0) spart[(size_t)rt * gridDim.x + ct] = red[0] + red[1] + red[2] + red[3];
}

constexpr size_t kFusedDotsSmem = sizeof(double) * (kFC * kFLD + kFC + kFR + 4 * kFR + 8);

__global__ void __launch_bounds__(256) fused_finalize_kernel(
    int n, int np, int cl, int nrt, int nct, const double* __restrict__ upart,
    const double* __restrict__ wpart, const double* __restrict__ spart,
    const double* __restrict__ tau_p, double* __restrict__ u, double* __restrict__ w,
    double* __restrict__ s_out) {
  if (*tau_p == 0.0) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= cl && idx < n) {
    double a = 0.0;
    for (int r = 0; r < nrt; ++r) a += upart[(size_t)r * n + idx];
    u[idx] = a;
  }
  if (idx < np) {
    double b = 0.0;
    for (int c = 0; c < nct; ++c) b += wpart[(size_t)c * np + idx];
    w[idx] = b;
  }
  if (blockIdx.x == 0) {
    __shared__ double red[256];
    double a = 0.0;
    for (int k = threadIdx.x; k < nrt * nct; k += blockDim.x) a += spart[k];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) *s_out = red[0];
  }
}

// Pass 2: A -= tau v u^T (rows >= r0) + tau w' v^T; thread (row, quarter)
// updates 32 columns with independent loads.
__global__ void __launch_bounds__(256) fused_update_kernel(
    double* __restrict__ A, int n, double* __restrict__ C, int ldc, int p, int r0, int cl,
    const double* __restrict__ vsrc, const double* __restrict__ tau_p,
    const double* __restrict__ u, const double* __restrict__ w, const double* __restrict__ s_p) {
  const double tau = *tau_p;
  if (tau == 0.0) return;
  __shared__ double vc_s[kFC];
  __shared__ double tu_s[kFC];
  const int tid = threadIdx.x;
  const int rt = blockIdx.y, ct = blockIdx.x;
  const int c0 = cl + ct * kFC;
  const int np = n + p;
  if (tid < kFC) {
    const int c = c0 + tid;
    vc_s[tid] = (c < n) ? vrow(c, r0, n, vsrc) : 0.0;
    tu_s[tid] = (c < n) ? tau * u[c] : 0.0;
  }
  __syncthreads();
  const int r = tid % kFR, qtr = tid / kFR;
  const int i = rt * kFR + r;
  if (i >= np) return;
  const double vi = vrow(i, r0, n, vsrc);
  const double twp = tau * (w[i] - tau * (*s_p) * vi);   // tau * w'_i
  const double lvi = (i >= r0 && i < n) ? vi : 0.0;       // left part only on rows >= r0
  const int cb = c0 + qtr * 32;
  const int cnt = min(32, n - cb);
  if (cnt <= 0) return;
  double* base = i < n ? A + i : C + (i - n);
  const size_t ld = i < n ? (size_t)n : (size_t)ldc;
  double a[32];
#pragma unroll
  for (int k = 0; k < 32; ++k)
    if (k < cnt) a[k] = base[(size_t)(cb + k) * ld];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < cnt) {
      const int cc = qtr * 32 + k;
      double v = fma(-lvi, tu_s[cc], a[k]);
      base[(size_t)(cb + k) * ld] = fma(-twp, vc_s[cc], v);
    }
  }
}

struct FusedWork {
  double* upart;
  double* wpart;
  double* spart;
  double* u;
  double* w;
  double* s;
};

inline cudaError_t launch_two_sided(double* A, int n, double* C, int ldc, int p, int r0, int cl,
                                    const double* vsrc, const double* tau, const FusedWork& fw,
                                    cudaStream_t st) {
  if (n - r0 <= 1) return cudaSuccess;
  const int np = n + p;
  const int nrt = (np + kFR - 1) / kFR;
  const int nct = (n - cl + kFC - 1) / kFC;
  dim3 grid(nct, nrt);
  fused_dots_kernel<<<grid, 256, kFusedDotsSmem, st>>>(A, n, C, ldc, p, r0, cl, vsrc, tau,
                                                       fw.upart, fw.wpart, fw.spart);
  count_launch();
  fused_finalize_kernel<<<(std::max(n, np) + 255) / 256, 256, 0, st>>>(
      n, np, cl, nrt, nct, fw.upart, fw.wpart, fw.spart, tau, fw.u, fw.w, fw.s);
  count_launch();
  fused_update_kernel<<<grid, 256, 0, st>>>(A, n, C, ldc, p, r0, cl, vsrc, tau, fw.u, fw.w, fw.s);
  count_launch();
  return cudaGetLastError();
}


// Frobenius norm^2 and trace of the structural part of H.
__global__ void hnorm_kernel(const double* __restrict__ H, int n, int m, double* __restrict__ out) {
  __shared__ double red[2][8];
  double s2 = 0.0, tr = 0.0;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * n;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    if (i <= j + m) {
      double v = H[idx];
      s2 = fma(v, v, s2);
      if (i == j) tr += v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_down_sync(0xffffffffu, s2, o);
    tr += __shfl_down_sync(0xffffffffu, tr, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s2;
    red[1][threadIdx.x >> 5] = tr;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += red[0][w]; b += red[1][w]; }
    atomicAdd(out, a);
    atomicAdd(out + 1, b);
  }
}

// Left application of one reflector to complex columns (for X = Q Xhat).
__global__ void __launch_bounds__(256) apply_left_complex_kernel(
    cd* __restrict__ X, long long ldx, int r0, int len, int ncols, const double* __restrict__ vsrc,
    const double* __restrict__ tau_p) {
  double tau = *tau_p;
  if (tau == 0.0) return;
  int lane = threadIdx.x & 31;
  int col = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (col >= ncols) return;
  cd* x = X + (size_t)col * ldx + r0;
  double dr = 0.0, di = 0.0;
  for (int i = lane; i < len; i += 32) {
    double v = i == 0 ? 1.0 : vsrc[i];
    dr = fma(v, x[i].x, dr);
    di = fma(v, x[i].y, di);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dr += __shfl_xor_sync(0xffffffffu, dr, o);
    di += __shfl_xor_sync(0xffffffffu, di, o);
  }
  dr *= tau;
  di *= tau;
  for (int i = lane; i < len; i += 32) {
    double v = i == 0 ? 1.0 : vsrc[i];
    x[i].x = fma(-v, dr, x[i].x);
    x[i].y = fma(-v, di, x[i].y);
  }
}

__global__ void copy_masked_kernel(const double* __restrict__ src, long long lds, int rows, int cols,
                                   int band, double* __restrict__ dst, long long ldd) {
  // dst(i, j) = src(i, j) if i <= j + band else 0
  long long total = (long long)rows * cols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx % rows), j = (int)(idx / rows);
    dst[i + (size_t)j * ldd] = (i <= j + band) ? src[i + (size_t)j * lds] : 0.0;
  }
}

__global__ void copy_cd_kernel(const cd* __restrict__ src, long long lds, int rows, int cols,
                               cd* __restrict__ dst, long long ldd) {
  long long total = (long long)rows * cols;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx % rows), j = (int)(idx / rows);
    dst[i + (size_t)j * ldd] = src[i + (size_t)j * lds];
  }
}

// Hhi = fl32(H), Hlo = fl32(H - Hhi) on and above the m-th subdiagonal; 0 below.
__global__ void split_h_kernel(const double* __restrict__ H, int n, int m, float* __restrict__ hi,
                               float* __restrict__ lo) {
  long long total = (long long)n * n;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int i = (int)(idx % n), j = (int)(idx / n);
    float a = 0.0f, b = 0.0f;
    if (i <= j + m) {
      double v = H[idx];
      a = (float)v;
      b = (float)(v - (double)a);
    }
    hi[idx] = a;
    lo[idx] = b;
  }
}

// One Householder reflector on the left of rows [r0, r0+len) of a's columns
// [c0, c1), where v lives at vsrc (vsrc[0] ignored, treated as 1).
inline cudaError_t launch_left(double* a, long long ld, int r0, int len, int c0, int c1,
                               const double* vsrc, const double* tau, cudaStream_t st) {
  if (c1 <= c0 || len <= 1) return cudaSuccess;
  long long warps = c1 - c0;
  int blocks = (int)((warps * 32 + 255) / 256);
  apply_left_kernel<<<blocks, 256, 0, st>>>(a, ld, r0, len, c0, c1, vsrc, tau);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

int reduce_fp64(Handle* h, const double* A, long long lda, const double* B, long long ldb,
                const double* C, long long ldc, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  const int ldct = p > 0 ? p : 1;
  SSV_CUDA_TRY(cudaMemcpy2DAsync(h->H, sizeof(double) * n, A, sizeof(double) * lda,
                                 sizeof(double) * n, n, cudaMemcpyDeviceToDevice, st));
  SSV_CUDA_TRY(cudaMemcpy2DAsync(h->R, sizeof(double) * n, B, sizeof(double) * ldb,
                                 sizeof(double) * n, m, cudaMemcpyDeviceToDevice, st));
  if (p > 0)
    SSV_CUDA_TRY(cudaMemcpy2DAsync(h->Ct, sizeof(double) * ldct, C, sizeof(double) * ldc,
                                   sizeof(double) * p, n, cudaMemcpyDeviceToDevice, st));
  SSV_CUDA_TRY(cudaFuncSetAttribute(fused_dots_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kFusedDotsSmem));
  // workspace of the two-sided reflector application
  const int np = n + p;
  const size_t nrt_max = (size_t)(np + kFR - 1) / kFR;
  const size_t nct_max = (size_t)(n + kFC - 1) / kFC;
  const size_t wbytes = sizeof(double) * (nrt_max * n + nct_max * np + nrt_max * nct_max + n + np + 1);
  double* wsp = nullptr;
  SSV_CUDA_TRY(cudaMallocAsync((void**)&wsp, wbytes, st));
  FusedWork fw;
  fw.upart = wsp;
  fw.wpart = fw.upart + nrt_max * n;
  fw.spart = fw.wpart + nct_max * np;
  fw.u = fw.spart + nrt_max * nct_max;
  fw.w = fw.u + n;
  fw.s = fw.w + np;

  int rc = SSV_OK;
  auto chk = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == SSV_OK) {
      set_cuda_error(e);
      rc = SSV_ECUDA;
    }
  };
  // Steps 1-2: QR of B; each reflector applied to the rest of B, and to A from
  // both sides and to C from the right (left part: all columns).
  h->kb = std::min(m, n - 1);
  for (int i = 0; i < h->kb && rc == SSV_OK; ++i) {
    int len = n - i;
    double* x = h->R + i + (size_t)i * n;
    house_kernel<<<1, kHouseThreads, 0, st>>>(x, len, h->tauB + i);
    count_launch();
    chk(cudaGetLastError());
    chk(launch_left(h->R, n, i, len, i + 1, m, x, h->tauB + i, st));
    chk(launch_two_sided(h->H, n, h->Ct, ldct, p, i, 0, x, h->tauB + i, fw, st));
  }
  // Steps 3-4: m-Hessenberg reduction of A, C <- C Q_A.  Reflector j acts on
  // rows/columns j+m .. n-1; its left part touches columns j+1 .. n-1.
  h->ka = std::max(0, n - m - 1);
  for (int j = 0; j < h->ka && rc == SSV_OK; ++j) {
    int r0 = j + m, len = n - r0;
    double* x = h->H + r0 + (size_t)j * n;
    house_kernel<<<1, kHouseThreads, 0, st>>>(x, len, h->tauA + j);
    count_launch();
    chk(cudaGetLastError());
    chk(launch_two_sided(h->H, n, h->Ct, ldct, p, r0, j + 1, x, h->tauA + j, fw, st));
  }
  h->has_q = 1;
  if (rc == SSV_OK) {
    chk(cudaMemsetAsync(h->hnorm2, 0, 2 * sizeof(double), st));
    hnorm_kernel<<<std::max(1, std::min(1024, (n * n + 255) / 256)), 256, 0, st>>>(h->H, n, m,
                                                                                  h->hnorm2);
    count_launch();
    chk(cudaGetLastError());
  }
  chk(cudaFreeAsync(wsp, st));
  return rc;
}

int apply_q_fp64(const Handle* h, int ncols, const double* Xhat, long long ldx, double* X,
                 long long ldX, cudaStream_t st) {
  const int n = h->n, m = h->m;
  if (ncols == 0) return SSV_OK;
  cd* Xc = reinterpret_cast<cd*>(X);
  if (X != Xhat) {
    int blocks = (int)std::min<long long>(4096, ((long long)n * ncols + 255) / 256);
    copy_cd_kernel<<<blocks, 256, 0, st>>>(reinterpret_cast<const cd*>(Xhat), ldx, n, ncols, Xc,
                                           ldX);
    count_launch();
    SSV_CUDA_TRY(cudaGetLastError());
  }
  int blocks = (int)(((long long)ncols * 32 + 255) / 256);
  // Q = Q_B Q_A = HB_0 .. HB_{kb-1} HA_0 .. HA_{ka-1}: apply the last reflector first.
  for (int j = h->ka - 1; j >= 0; --j) {
    int r0 = j + m, len = n - r0;
    apply_left_complex_kernel<<<blocks, 256, 0, st>>>(Xc, ldX, r0, len, ncols,
                                                      h->H + r0 + (size_t)j * n, h->tauA + j);
    count_launch();
  }
  for (int i = h->kb - 1; i >= 0; --i) {
    int len = n - i;
    apply_left_complex_kernel<<<blocks, 256, 0, st>>>(Xc, ldX, i, len, ncols,
                                                      h->R + i + (size_t)i * n, h->tauB + i);
    count_launch();
  }
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

int load_reduced(Handle* h, const double* H, long long ldh, const double* R, long long ldr,
                 const double* Ct, long long ldc, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  int blocks = (int)std::min<long long>(4096, ((long long)n * n + 255) / 256);
  copy_masked_kernel<<<blocks, 256, 0, st>>>(H, ldh, n, n, m, h->H, n);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  blocks = (int)std::min<long long>(4096, ((long long)n * m + 255) / 256);
  copy_masked_kernel<<<blocks, 256, 0, st>>>(R, ldr, n, m, 0, h->R, n);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  if (p > 0)
    SSV_CUDA_TRY(cudaMemcpy2DAsync(h->Ct, sizeof(double) * p, Ct, sizeof(double) * ldc,
                                   sizeof(double) * p, n, cudaMemcpyDeviceToDevice, st));
  h->kb = 0;
  h->ka = 0;
  h->has_q = 0;
  SSV_CUDA_TRY(cudaMemsetAsync(h->hnorm2, 0, 2 * sizeof(double), st));
  hnorm_kernel<<<std::max(1, std::min(1024, (n * n + 255) / 256)), 256, 0, st>>>(h->H, n, m,
                                                                                h->hnorm2);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

int split_h(Handle* h, cudaStream_t st) {
  const int n = h->n;
  int blocks = (int)std::min<long long>(8192, ((long long)n * n + 255) / 256);
  split_h_kernel<<<blocks, 256, 0, st>>>(h->H, n, h->m, h->Hhi, h->Hlo);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

int get_reduced(const Handle* h, double* H, long long ldh, double* R, long long ldr, double* Ct,
                long long ldc, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  if (H) {
    int blocks = (int)std::min<long long>(4096, ((long long)n * n + 255) / 256);
    copy_masked_kernel<<<blocks, 256, 0, st>>>(h->H, n, n, n, m, H, ldh);
    count_launch();
    SSV_CUDA_TRY(cudaGetLastError());
  }
  if (R) {
    int blocks = (int)std::min<long long>(4096, ((long long)n * m + 255) / 256);
    copy_masked_kernel<<<blocks, 256, 0, st>>>(h->R, n, n, m, 0, R, ldr);
    count_launch();
    SSV_CUDA_TRY(cudaGetLastError());
  }
  if (Ct && p > 0) {
    SSV_CUDA_TRY(cudaMemcpy2DAsync(Ct, sizeof(double) * ldc, h->Ct, sizeof(double) * p,
                                   sizeof(double) * p, n, cudaMemcpyDeviceToDevice, st));
  }
  return SSV_OK;
}

}  // namespace ssv
