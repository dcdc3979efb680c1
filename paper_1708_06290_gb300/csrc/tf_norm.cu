// ||C (sigma I - A)^{-1} B||_2 for every shift: the function whose level sets
// are the structured pseudospectrum of (A, B, C) (Sec. 1, the set of z with
// ||C (zI - A)^{-1} B||_2 >= 1/eps).
//
// The transfer function G(sigma) (p x m) comes from the shifted solve in any
// precision; its largest singular value is sqrt(lambda_max(M)) with
// M = G^H G (m <= p) or G G^H (m > p), k x k Hermitian, k = min(m, p) <= 32.
// One warp per shift runs cyclic two-sided Jacobi on M in shared memory: for
// the pair (a, b) with M(a, b) = |g| e^{i phi}, the rotation
//   J = [[c, s], [-s e^{-i phi}, c e^{-i phi}]],  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
//   tau = (M(b, b) - M(a, a)) / (2 |g|),  c = 1 / sqrt(1 + t^2),  s = t c
// zeroes M(a, b) in J^H M J (the real symmetric Jacobi rotation after the
// diagonal phase change diag(1, e^{-i phi})); lanes update the k entries of
// columns a, b and then of rows a, b.  Sweeps stop when the off-diagonal
// mass is below 1e-30 of the diagonal's (at most 40 sweeps).
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kMaxK = 32;
constexpr int kLdM = kMaxK + 1;

__global__ void __launch_bounds__(32 * kWarpsPerBlock) tf_norm_kernel(const cd* __restrict__ G,
                                                                      long long ldg, int p, int m,
                                                                      int s, double* __restrict__ norms) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int sh = blockIdx.x * kWarpsPerBlock + wib;
  if (sh >= s) return;  // warp-uniform
  cd* M = reinterpret_cast<cd*>(smem_raw) + (size_t)wib * kMaxK * kLdM;
  const int k = min(m, p);
  const cd* g = G + (size_t)sh * m * ldg;  // G(i, j) = g[i + j * ldg], p x m
  // M = G^H G (k = m) or G G^H (k = p)
  for (int e = lane; e < k * k; e += 32) {
    const int a = e % k, b = e / k;
    cd acc = mkcd(0.0, 0.0);
    if (m <= p) {
      for (int i = 0; i < p; ++i) {
        const cd x = g[i + (size_t)a * ldg], y = g[i + (size_t)b * ldg];
        acc = cfma(mkcd(x.x, -x.y), y, acc);
      }
    } else {
      for (int j = 0; j < m; ++j) {
        const cd x = g[a + (size_t)j * ldg], y = g[b + (size_t)j * ldg];
        acc = cfma(x, mkcd(y.x, -y.y), acc);
      }
    }
    M[a + b * kLdM] = acc;
  }
  __syncwarp();
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dg = 0.0;
    for (int e = lane; e < k * k; e += 32) {
      const int a = e % k, b = e / k;
      const cd v = M[a + b * kLdM];
      const double v2 = v.x * v.x + v.y * v.y;
      if (a == b) dg += v2;
      else off += v2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dg += __shfl_xor_sync(0xffffffffu, dg, o);
    }
    if (!(off > 1e-30 * dg)) break;  // also stops on NaN
    for (int a = 0; a < k - 1; ++a) {
      for (int b = a + 1; b < k; ++b) {
        const cd gab = M[a + b * kLdM];
        const double ag = hypot(gab.x, gab.y);
        if (ag == 0.0) continue;  // warp-uniform (same smem value)
        const cd ph = mkcd(gab.x / ag, gab.y / ag);  // e^{i phi}
        const cd phc = mkcd(ph.x, -ph.y);
        const double tau = (M[b + b * kLdM].x - M[a + a * kLdM].x) / (2.0 * ag);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t), sn = t * c;
        __syncwarp();
        // columns: [x_a, x_b] <- [c x_a - s e^{-i phi} x_b, s x_a + c e^{-i phi} x_b]
        if (lane < k) {
          const cd xa = M[lane + a * kLdM], xb = M[lane + b * kLdM];
          const cd pxb = cmul(phc, xb);
          M[lane + a * kLdM] = mkcd(c * xa.x - sn * pxb.x, c * xa.y - sn * pxb.y);
          M[lane + b * kLdM] = mkcd(sn * xa.x + c * pxb.x, sn * xa.y + c * pxb.y);
        }
        __syncwarp();
        // rows: [y_a; y_b] <- [c y_a - s e^{i phi} y_b; s y_a + c e^{i phi} y_b]
        if (lane < k) {
          const cd ya = M[a + lane * kLdM], yb = M[b + lane * kLdM];
          const cd pyb = cmul(ph, yb);
          M[a + lane * kLdM] = mkcd(c * ya.x - sn * pyb.x, c * ya.y - sn * pyb.y);
          M[b + lane * kLdM] = mkcd(sn * ya.x + c * pyb.x, sn * ya.y + c * pyb.y);
        }
        __syncwarp();
      }
    }
  }
  double lmax = 0.0;
  for (int a = lane; a < k; a += 32) lmax = fmax(lmax, M[a + a * kLdM].x);
  for (int o = 16; o > 0; o >>= 1) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  // a NaN anywhere in G propagates (fmax would drop it)
  double any_nan = 0.0;
  for (int e = lane; e < k * k; e += 32) {
    const cd v = M[(e % k) + (e / k) * kLdM];
    if (!(v.x == v.x) || !(v.y == v.y)) any_nan = 1.0;
  }
  for (int o = 16; o > 0; o >>= 1) any_nan = fmax(any_nan, __shfl_xor_sync(0xffffffffu, any_nan, o));
  if (lane == 0) norms[sh] = any_nan != 0.0 ? __longlong_as_double(0x7ff8000000000000LL) : sqrt(lmax);
}

}  // namespace

int tf_norm2(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* norms,
             int* status, cudaStream_t st) {
  const int m = h->m, p = h->p;
  if (s == 0) return SSV_OK;
  const int k = std::min(m, p);
  if (k < 1 || k > kMaxK) return SSV_ENOTSUP;
  ssv_opts og = *o;
  og.mode = SSV_G;
  cd* G = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&G, sizeof(cd) * (size_t)p * m * s, st));
  int rc = og.precision == SSV_MIXED
               ? solve_mixed(h, s, shifts, &og, reinterpret_cast<double*>(G), p, status, nullptr, st)
           : og.precision == SSV_SPLIT
               ? solve_split(h, s, shifts, SSV_G, reinterpret_cast<double*>(G), p, status, nullptr, st)
               : solve_fp64(h, s, shifts, &og, reinterpret_cast<double*>(G), p, status, nullptr, st);
  if (rc == SSV_OK) {
    const size_t smem = sizeof(cd) * kWarpsPerBlock * kMaxK * kLdM;
    cudaError_t e = cudaFuncSetAttribute(tf_norm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e == cudaSuccess) {
      tf_norm_kernel<<<(s + kWarpsPerBlock - 1) / kWarpsPerBlock, 32 * kWarpsPerBlock, smem, st>>>(
          G, p, p, m, s, norms);
      count_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = SSV_ECUDA;
    }
  }
  cudaError_t e2 = cudaFreeAsync(G, st);
  if (e2 != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e2);
    rc = SSV_ECUDA;
  }
  return rc;
}

}  // namespace ssv
