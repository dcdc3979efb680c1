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

}  // namespace

int reduce_fp64(Handle* h, const double* A, long long lda, const double* B, long long ldb,
                const double* C, long long ldc, int arith, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  const int ldct = p > 0 ? p : 1;
  SSV_CUDA_TRY(cudaMemcpy2DAsync(h->H, sizeof(double) * n, A, sizeof(double) * lda,
                                 sizeof(double) * n, n, cudaMemcpyDeviceToDevice, st));
  SSV_CUDA_TRY(cudaMemcpy2DAsync(h->R, sizeof(double) * n, B, sizeof(double) * ldb,
                                 sizeof(double) * n, m, cudaMemcpyDeviceToDevice, st));
  if (p > 0)
    SSV_CUDA_TRY(cudaMemcpy2DAsync(h->Ct, sizeof(double) * ldct, C, sizeof(double) * ldc,
                                   sizeof(double) * p, n, cudaMemcpyDeviceToDevice, st));
  // Steps 1-4 of Algorithm 1: one persistent cooperative kernel on the FP64
  // pipe, or the two-level blocked form with its products on the tensor cores
  int rc = arith == SSV_REDUCE_TENSOR ? reduce_tc(h, st) : reduce_persistent(h, st);
  if (rc != SSV_OK) return rc;
  h->has_q = 1;
  SSV_CUDA_TRY(cudaMemsetAsync(h->hnorm2, 0, 2 * sizeof(double), st));
  hnorm_kernel<<<std::max(1, std::min(1024, (n * n + 255) / 256)), 256, 0, st>>>(h->H, n, m,
                                                                                h->hnorm2);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
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
