// Normwise backward error of computed solutions Xhat of (H - sigma I) Xhat = R:
//   ||(H - sigma I) Xhat - R||_F / (||H - sigma I||_F ||Xhat||_F + ||R||_F),
// all in FP64.  Only the structural part of H (rows <= column + m) is read.
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {

namespace {

constexpr int kRows = 128;

template <int MAXM>
__global__ void __launch_bounds__(kRows) residual_kernel(int n, int m, const double* __restrict__ H,
                                                         const double* __restrict__ R,
                                                         const cd* __restrict__ shifts,
                                                         const cd* __restrict__ X, long long ldx,
                                                         double* __restrict__ acc,
                                                         const int* __restrict__ mask) {
  const int sh = blockIdx.y;
  if (mask != nullptr && mask[sh] == 0) return;
  const int i = blockIdx.x * kRows + threadIdx.x;
  const cd sigma = shifts[sh];
  const cd* Xs = X + (size_t)sh * m * ldx;
  __shared__ double red[2][kRows / 32];
  double e2 = 0.0, x2 = 0.0;
  const int jlo = max(0, (int)(blockIdx.x * kRows) - m);
  if (i < n) {
    cd e[MAXM];
#pragma unroll
    for (int q = 0; q < MAXM; ++q) e[q] = mkcd(0.0, 0.0);
    for (int j = jlo; j < n; ++j) {
      const double hij = (j >= i - m) ? H[i + (size_t)j * n] : 0.0;
#pragma unroll
      for (int q = 0; q < MAXM; ++q) {
        if (q < m) {
          const cd x = Xs[j + (size_t)q * ldx];
          e[q].x = fma(hij, x.x, e[q].x);
          e[q].y = fma(hij, x.y, e[q].y);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < MAXM; ++q) {
      if (q < m) {
        const cd x = Xs[i + (size_t)q * ldx];
        cd v = cfms(sigma, x, e[q]);
        if (i <= q) v.x -= R[i + (size_t)q * n];
        e2 = fma(v.x, v.x, fma(v.y, v.y, e2));
        x2 = fma(x.x, x.x, fma(x.y, x.y, x2));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    e2 += __shfl_down_sync(0xffffffffu, e2, o);
    x2 += __shfl_down_sync(0xffffffffu, x2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = e2;
    red[1][threadIdx.x >> 5] = x2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int w = 0; w < kRows / 32; ++w) { a += red[0][w]; b += red[1][w]; }
    atomicAdd(acc + 2 * sh, a);
    atomicAdd(acc + 2 * sh + 1, b);
  }
}

__global__ void residual_finish_kernel(int n, int m, int s, const double* __restrict__ hn,
                                       const double* __restrict__ R, const cd* __restrict__ shifts,
                                       const double* __restrict__ acc, double* __restrict__ resid,
                                       const int* __restrict__ mask) {
  int sh = blockIdx.x * blockDim.x + threadIdx.x;
  if (sh >= s) return;
  if (mask != nullptr && mask[sh] == 0) return;
  double r2 = 0.0;
  for (int q = 0; q < m; ++q)
    for (int i = 0; i <= q && i < n; ++i) r2 = fma(R[i + (size_t)q * n], R[i + (size_t)q * n], r2);
  const cd sg = shifts[sh];
  double m2 = hn[0] - 2.0 * sg.x * hn[1] + (double)n * (sg.x * sg.x + sg.y * sg.y);
  m2 = fmax(m2, 0.0);
  double den = sqrt(m2) * sqrt(acc[2 * sh + 1]) + sqrt(r2);
  // a NaN denominator (non-finite Xhat) must not read as a zero backward error
  resid[sh] = den > 0 ? sqrt(acc[2 * sh]) / den : (den == den ? 0.0 : den);
}

template <int MAXM>
int launch(const Handle* h, int s, const double* shifts, const double* Xhat, long long ldx,
           double* resid, double* acc, const int* mask, cudaStream_t st) {
  dim3 grid((h->n + kRows - 1) / kRows, s);
  residual_kernel<MAXM><<<grid, kRows, 0, st>>>(h->n, h->m, h->H, h->R,
                                                reinterpret_cast<const cd*>(shifts),
                                                reinterpret_cast<const cd*>(Xhat), ldx, acc, mask);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

}  // namespace

int backward_error_fp64(const Handle* h, int s, const double* shifts, const double* Xhat,
                        long long ldx, double* resid, cudaStream_t st) {
  return backward_error_fp64_masked(h, s, shifts, Xhat, ldx, resid, nullptr, st);
}

int backward_error_fp64_masked(const Handle* h, int s, const double* shifts, const double* Xhat,
                               long long ldx, double* resid, const int* mask, cudaStream_t st) {
  if (s == 0) return SSV_OK;
  double* acc = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&acc, sizeof(double) * 2 * s, st));
  int rc = SSV_OK;
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 2 * s, st);
  if (e != cudaSuccess) { set_cuda_error(e); rc = SSV_ECUDA; }
  const int m = h->m;
  if (rc == SSV_OK) {
    if (m <= 1) rc = launch<1>(h, s, shifts, Xhat, ldx, resid, acc, mask, st);
    else if (m <= 2) rc = launch<2>(h, s, shifts, Xhat, ldx, resid, acc, mask, st);
    else if (m <= 4) rc = launch<4>(h, s, shifts, Xhat, ldx, resid, acc, mask, st);
    else if (m <= 8) rc = launch<8>(h, s, shifts, Xhat, ldx, resid, acc, mask, st);
    else if (m <= 16) rc = launch<16>(h, s, shifts, Xhat, ldx, resid, acc, mask, st);
    else rc = launch<32>(h, s, shifts, Xhat, ldx, resid, acc, mask, st);
  }
  if (rc == SSV_OK) {
    residual_finish_kernel<<<(s + 127) / 128, 128, 0, st>>>(h->n, m, s, h->hnorm2, h->R,
                                                            reinterpret_cast<const cd*>(shifts),
                                                            acc, resid, mask);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) { set_cuda_error(e); rc = SSV_ECUDA; }
  }
  e = cudaFreeAsync(acc, st);
  if (e != cudaSuccess && rc == SSV_OK) { set_cuda_error(e); rc = SSV_ECUDA; }
  return rc;
}

}  // namespace ssv
