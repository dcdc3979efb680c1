// Controller-Hessenberg reduction (Algorithm 1, Sec. 2) as ONE persistent
// cooperative kernel, blocked by mini-blocks of reflectors (the m-column
// mini-blocks of Algorithms 2/3).
//
// Why mini-blocks of width w <= m need no per-column matrix-vector product:
// the reflector of column j acts on rows/columns j+m .. n-1, so applying it
// from the right never touches columns j .. j+m-1.  The w reflectors of the
// mini-block j0 .. j0+w-1 are therefore the Householder QR of the tall panel
// A(j0+m : n-1, j0 : j0+w-1) alone.  With their compact WY form
// Q = I - V T V^T (T upper triangular, LAPACK's forward column-wise form):
//
//   phase B (all blocks, row strips):  Y = A_ext(:, r0:) V T   (A_ext = [A; C])
//   phase C, bottom (column strips of rows r0 .. n-1):
//       A(r0:, r0:) -= Y V^T                        (right update, A Q)
//       W  = V^T A(r0:, lc:),  A(r0:, lc:) -= V (T^T W)   (left update, Q^T A)
//   phase C, top (2D tiles of the rows above r0 and of C):
//       A_ext(top, r0:) -= Y V^T                    (right update, A Q and C Q)
//   phase C's two kinds of work are split between blocks by multiply-add count.
//
// with r0 = j0 + m and lc = j0 + w, w = min(m, 8).  Every phase is a
// multiply-add stream on the FP64 pipe; the loops are instantiated for
// w = 1, 2, 4, 8.  The QR of B (Step 1) is one panel of width m; its
// reflectors are applied to A and C in groups of at most kW with r0 = group
// start and lc = 0.
//
// Look-ahead: in phase C block 0 owns exactly the columns of the NEXT panel;
// after updating them it factors that panel while the other blocks finish
// their strips, so each mini-block costs two grid barriers (after phase B and
// after phase C + panel).
//
// The barrier is the library's own: it spins with a bounded iteration count
// and, if the count runs out, raises an error flag so every block returns and
// the host reports SSV_ETIMEOUT.  The cooperative launch guarantees that all
// blocks are resident, so in normal operation every wait ends.
//
// Data written by other blocks during the kernel is always read with __ldcg
// (L2; the SM's L1 is not coherent across SMs).
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {

namespace {

constexpr int kT = 512;          // threads per block (one block per SM)
constexpr int kWarps = kT / 32;
constexpr int kW = 8;            // maximum reflectors per block step
constexpr int kWA = 8;           // reflectors per A mini-block (<= m): balances the panel
                                 // block's look-ahead work against the others' strips
constexpr int kVCW = 1024;       // V rows x width staged per chunk (phases B and C, pass 2)
constexpr int kVLD = kW + 1;     // padded row stride of staged V (conflict-free)
constexpr int kRS = 64;          // maximum rows per phase-B sub-strip
constexpr int kSCmax = 32;       // strip columns per phase-C sub-chunk
constexpr int kTR = 64;          // rows of a phase-C top tile
constexpr int kTC = 64;          // columns of a phase-C top tile
constexpr int kMaxDots = 16;     // dot products reduced together in the panel QR (>= 2 kW - 1)
constexpr unsigned long long kBarrierSpins = 1ull << 28;  // ~10 s of 32 ns naps

// shared-memory layout (doubles)
constexpr int kSmVc = 2 * kVCW;                 // staged V chunk: (1024 / w) rows, stride <= w + 1
constexpr int kSmPart = kT * kW;                // phase B: partial sums (CG x RS x kW <= kT x kW)
constexpr int kSmAV = kRS * kW;                 // phase B: reduced A V rows
constexpr int kSmT = kW * kW;                   // T of the current step
constexpr int kSmB = kSmVc + kSmPart + kSmAV;
constexpr int kSmVs = kSCmax * kVLD;            // phase C: V rows of the sub-chunk's columns
constexpr int kSmWs = kW * kSCmax;              // phase C: W, then Z = T^T W
constexpr int kSmC = kSmVs + 2 * kSmWs + kSmVc;   // + staged V rows (pass 2)
constexpr int kSmTop = (kTR + kTC) * kVLD;       // phase C top tile: Y and V rows
constexpr int kSmQ = kWarps * kMaxDots + kMaxDots + kSmT + 8;   // panel QR
constexpr int kSmDoubles = kSmT + std::max(std::max(kSmB, kSmTop), std::max(kSmC, kSmQ));

struct RedArgs {
  double* H;
  double* R;
  double* Ct;
  double* tauA;
  double* tauB;
  int n, m, p, ldct, kb, ka, wa;
  double* VB;      // n x kb rows of the B reflectors (row-major, ld kb)
  double* TB;      // ceil(kb / kW) blocks of kW x kW
  double* VA;      // 2 x (n x kW): rows of the current / next mini-block's V
  double* TA;      // 2 x (kW x kW)
  double* Y;       // (n + p) x kW
  unsigned* bar;   // [0] arrivals, [1] generation
  int* err;        // 1 after a barrier timed out
};

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

// Sum of `cnt` (<= kMaxDots) per-thread values over the block -> out[0..cnt).
__device__ void block_sum_vec(const double* acc, int cnt, double* red, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kMaxDots; ++q) {
    if (q < cnt) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[warp * kMaxDots + q] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < cnt) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red[w * kMaxDots + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Householder QR of the L x wc panel P (column-major, leading dimension ld)
// with wp <= wc reflectors (the columns wp .. wc-1 only receive them),
// L - k >= 2 for every reflector k < wp.  Reflector k: beta on the diagonal,
// v(k+1:) below it (v(k) = 1), tau[k]; the rows of V (unit lower trapezoidal,
// explicit ones and zeros) go to Vout (row-major, ld ldv) and the triangular
// factor of each group of wg consecutive reflectors to Tout (kW x kW blocks,
// row-major).  Rows are owned by thread (row mod kT) throughout.
__device__ void panel_qr(double* P, size_t ld, int L, int wp, int wc, int wg, double* tau,
                         double* Vout, int ldv, double* Tout, double* sm) {
  double* red = sm;                          // kWarps x kMaxDots
  double* dots = red + kWarps * kMaxDots;    // kMaxDots
  double* Tl = dots + kMaxDots;              // kW x kW
  double* misc = Tl + kSmT;                  // [0] scal, [1] tau
  const int tid = threadIdx.x;
  for (int k = 0; k < wp; ++k) {
    double* x = P + (size_t)k * ld;
    const int g0 = (k / wg) * wg;
    const int jj = k - g0;
    // (a) norm of x(k+1:L) and the reflector
    {
      double ss = 0.0;
      for (int i = k + 1 + ((tid - (k + 1)) % kT + kT) % kT; i < L; i += kT) {
        const double xi = __ldcg(x + i);
        ss = fma(xi, xi, ss);
      }
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      if ((tid & 31) == 0) red[tid >> 5] = ss;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kWarps; ++w) t += red[w];
        dots[0] = t;
      }
      __syncthreads();
    }
    if (tid == 0) {
      const double v = dots[0];
      const double alpha = __ldcg(x + k);
      double tk = 0.0, scal = 0.0;
      if (v != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, v));
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        tk = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
        x[k] = beta;
      }
      tau[k] = tk;
      misc[0] = scal;
      misc[1] = tk;
    }
    __syncthreads();
    const double scal = misc[0], tk = misc[1];
    // (b) v(k+1:) = x(k+1:) * scal   (own rows)
    const int ifirst = k + ((tid - k) % kT + kT) % kT;  // first own row >= k
    if (scal != 0.0)
      for (int i = ifirst; i < L; i += kT)
        if (i > k) x[i] = __ldcg(x + i) * scal;
    // (c) dots: d_q = v^T P(:, q) for q = k+1 .. wc-1, then z_j = V(:, j)^T v
    //     for j = g0 .. jj-1 (same group), in batches of kMaxDots
    const int nrest = wc - 1 - k;
    const int nd = nrest + jj;
    double zloc[kW];
    for (int b0 = 0; b0 < nd; b0 += kMaxDots) {
      const int cnt = min(kMaxDots, nd - b0);
      double acc[kMaxDots];
#pragma unroll
      for (int q = 0; q < kMaxDots; ++q) acc[q] = 0.0;
      for (int i = ifirst; i < L; i += kT) {
        const double vi = i == k ? 1.0 : __ldcg(x + i);
#pragma unroll
        for (int q = 0; q < kMaxDots; ++q) {
          if (q < cnt) {
            const int e = b0 + q;
            const int col = e < nrest ? k + 1 + e : g0 + (e - nrest);
            acc[q] = fma(vi, __ldcg(P + i + (size_t)col * ld), acc[q]);
          }
        }
      }
      block_sum_vec(acc, cnt, red, dots);
      // (d) update the remaining panel columns of this batch; keep the z's
      for (int q = 0; q < cnt; ++q) {
        const int e = b0 + q;
        if (e < nrest) {
          const int col = k + 1 + e;
          const double td = tk * dots[q];
          if (td != 0.0) {
            double* pc = P + (size_t)col * ld;
            for (int i = ifirst; i < L; i += kT) {
              const double vi = i == k ? 1.0 : __ldcg(x + i);
              pc[i] = fma(-td, vi, __ldcg(pc + i));
            }
          }
        } else if (tid == 0) {
          zloc[e - nrest] = dots[q];
        }
      }
      __syncthreads();
    }
    // (e) T(0:jj, jj) = -tau T(0:jj, 0:jj) z,  T(jj, jj) = tau
    if (tid == 0) {
      for (int r = 0; r < jj; ++r) {
        double s = 0.0;
        for (int c = r; c < jj; ++c) s = fma(Tl[r * kW + c], zloc[c], s);
        Tl[r * kW + jj] = -tk * s;
      }
      for (int r = jj + 1; r < kW; ++r) Tl[r * kW + jj] = 0.0;
      Tl[jj * kW + jj] = tk;
      if (jj == wg - 1 || k == wp - 1) {
        double* To = Tout + (size_t)(k / wg) * kSmT;
        for (int e = 0; e < kSmT; ++e) {
          const int r = e / kW, c = e % kW;
          To[e] = (r <= jj && c <= jj) ? Tl[e] : 0.0;
        }
      }
    }
    __syncthreads();
  }
  // dense rows of V
  for (long long o = tid; o < (long long)L * wp; o += kT) {
    const int i = (int)(o / wp), k = (int)(o % wp);
    const double v = i < k ? 0.0 : (i == k ? 1.0 : __ldcg(P + i + (size_t)k * ld));
    Vout[(size_t)i * ldv + k] = v;
  }
  __syncthreads();
}

// Row i of A_ext = [A; C]: base pointer and column stride.
__device__ __forceinline__ double* ext_row(const RedArgs& a, int i, size_t* ld) {
  if (i < a.n) {
    *ld = (size_t)a.n;
    return a.H + i;
  }
  *ld = (size_t)a.ldct;
  return a.Ct + (i - a.n);
}

// Phase B, rows [i0, i1) of A_ext: Y = A_ext(rows, r0:n) V T.  W >= w is the
// compile-time width (V and T are zero beyond w).
template <int W>
__device__ void phase_b(const RedArgs& a, int r0, int w, const double* __restrict__ V, int ldv,
                        const double* __restrict__ Ts, double* sm) {
  constexpr int VC = kVCW / W, VLD = W == 1 ? 1 : W + 1;
  const int n = a.n, np = a.n + a.p;
  double* Vc = sm;
  double* part = Vc + kSmVc;
  double* AV = part + kSmPart;
  const int tid = threadIdx.x;
  const int i0 = (int)(((long long)np * blockIdx.x) / gridDim.x);
  const int i1 = (int)(((long long)np * (blockIdx.x + 1)) / gridDim.x);
  for (int rs0 = i0; rs0 < i1; rs0 += kRS) {
    const int RS = min(kRS, i1 - rs0);
    const int CG = kT / RS;
    const int r = tid % RS, g = tid / RS;
    const bool act = g < CG;
    size_t ld = 0;
    const double* base = ext_row(a, rs0 + r, &ld);
    double acc[W];
#pragma unroll
    for (int k = 0; k < W; ++k) acc[k] = 0.0;
    for (int cb = r0; cb < n; cb += VC) {
      const int cnt = min(VC, n - cb);
      __syncthreads();
      for (int e = tid; e < cnt * W; e += kT) {
        const int q = e / W, k = e % W;
        Vc[q * VLD + k] = k < w ? __ldcg(V + (size_t)(cb - r0 + q) * ldv + k) : 0.0;
      }
      __syncthreads();
      if (act) {
        for (int q = g; q < cnt; q += CG) {
          const double x = __ldcg(base + (size_t)(cb + q) * ld);
          const double* vq = Vc + q * VLD;
#pragma unroll
          for (int k = 0; k < W; ++k) acc[k] = fma(x, vq[k], acc[k]);
        }
      }
    }
    if (act) {
#pragma unroll
      for (int k = 0; k < W; ++k) part[(g * RS + r) * W + k] = acc[k];
    }
    __syncthreads();
    for (int e = tid; e < RS * W; e += kT) {
      const int rr = e / W, k = e % W;
      double s = 0.0;
      for (int gg = 0; gg < CG; ++gg) s += part[(gg * RS + rr) * W + k];
      AV[rr * W + k] = s;
    }
    __syncthreads();
    for (int e = tid; e < RS * W; e += kT) {
      const int rr = e / W, k = e % W;
      double s = 0.0;
      for (int j = 0; j <= k; ++j) s = fma(AV[rr * W + j], Ts[j * kW + k], s);
      a.Y[(size_t)(rs0 + rr) * kW + k] = s;
    }
    __syncthreads();
  }
}

// Columns per phase-C sub-chunk: two per warp in pass 2.
template <int W>
struct SubChunk {
  static constexpr int kCols = 32;
  static constexpr int kPerWarp = kCols / kWarps;
};

// V rows (c - r0) of the columns cc .. cc+nc-1 into Vs (zero for columns < r0).
template <int W>
__device__ void stage_vcols(const double* __restrict__ V, int ldv, int r0, int w, int cc, int nc,
                            double* Vs) {
  __syncthreads();
  for (int e = threadIdx.x; e < SubChunk<W>::kCols * W; e += kT) {
    const int q = e / W, k = e % W;
    const int c = cc + q;
    Vs[q * kVLD + k] = (q < nc && c >= r0 && k < w) ? __ldcg(V + (size_t)(c - r0) * ldv + k) : 0.0;
  }
  __syncthreads();
}

// Right update A(i, c) -= Y(i, :) V(c - r0, :)^T for the rows i in [i0, i1)
// (all < n) and the staged columns q in [q0, nc) of the sub-chunk.
template <int W>
__device__ void right_rows(const RedArgs& a, int i0, int i1, int cc, int q0, int nc,
                           const double* Vs) {
  const int n = a.n;
  for (int i = i0 + threadIdx.x; i < i1; i += kT) {
    double y[W];
#pragma unroll
    for (int k = 0; k < W; ++k) y[k] = __ldcg(a.Y + (size_t)i * kW + k);
    double* base = a.H + i;
    for (int q = q0; q < nc; ++q) {
      double* px = base + (size_t)(cc + q) * n;
      double x = __ldcg(px);
      const double* vq = Vs + q * kVLD;
#pragma unroll
      for (int k = 0; k < W; ++k) x = fma(-y[k], vq[k], x);
      *px = x;
    }
  }
}

// Phase C, bottom part: columns [c0, c1) (all >= lc), rows r0 .. n-1:
// right update (columns >= r0), W = V^T A, left update with Z = T^T W.
template <int W>
__device__ void phase_c_bottom(const RedArgs& a, int r0, int w, const double* __restrict__ V,
                               int ldv, const double* __restrict__ Ts, int c0, int c1, double* sm) {
  constexpr int VC = kVCW / W, VLD = W == 1 ? 1 : W + 1;
  const int n = a.n;
  double* Vs = sm;
  double* Ws = Vs + kSmVs;
  double* Zs = Ws + kSmWs;
  double* Vc = Zs + kSmWs;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int SC = SubChunk<W>::kCols, CPW = SubChunk<W>::kPerWarp;
  const int nsub = (c1 - c0 + SC - 1) / SC;
  for (int sc = 0; sc < nsub; ++sc) {
    const int cc = c0 + (int)(((long long)(c1 - c0) * sc) / nsub);
    const int nc = c0 + (int)(((long long)(c1 - c0) * (sc + 1)) / nsub) - cc;
    stage_vcols<W>(V, ldv, r0, w, cc, nc, Vs);
    // pass 1: right update of rows r0 .. n-1
    const int qr = max(0, r0 - cc);
    if (qr < nc) right_rows<W>(a, r0, n, cc, qr, nc, Vs);
    // pass 2: W(:, q) = V^T A(r0:n, cc + q); warp owns columns warp + j * 16,
    // V rows staged per chunk of VC rows
    bool has[CPW];
    const double* pc[CPW];
    double acc[CPW][W];
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      const int q = warp + j * kWarps;
      has[j] = q < nc;
      pc[j] = a.H + (size_t)(cc + (has[j] ? q : 0)) * n;
#pragma unroll
      for (int k = 0; k < W; ++k) acc[j][k] = 0.0;
    }
    for (int ib = r0; ib < n; ib += VC) {
      const int cnt = min(VC, n - ib);
      __syncthreads();
      for (int e = tid; e < cnt * W; e += kT) {
        const int q = e / W, k = e % W;
        Vc[q * VLD + k] = k < w ? __ldcg(V + (size_t)(ib - r0 + q) * ldv + k) : 0.0;
      }
      __syncthreads();
      if (has[0]) {
        for (int q = lane; q < cnt; q += 32) {
          double x[CPW];
#pragma unroll
          for (int j = 0; j < CPW; ++j) x[j] = has[j] ? __ldcg(pc[j] + ib + q) : 0.0;
          const double* vq = Vc + q * VLD;
#pragma unroll
          for (int k = 0; k < W; ++k) {
            const double v = vq[k];
#pragma unroll
            for (int j = 0; j < CPW; ++j) acc[j][k] = fma(v, x[j], acc[j][k]);
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CPW; ++j) {
      if (has[j]) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          double u = acc[j][k];
          for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
          if (lane == 0) Ws[k * kSCmax + warp + j * kWarps] = u;
        }
      }
    }
    __syncthreads();
    // Z = T^T W
    for (int e = tid; e < W * nc; e += kT) {
      const int k = e / nc, q = e % nc;
      double s = 0.0;
      for (int j = 0; j <= k; ++j) s = fma(Ts[j * kW + k], Ws[j * kSCmax + q], s);
      Zs[k * kSCmax + q] = s;
    }
    __syncthreads();
    // pass 3: left update A(i, c) -= V(i - r0, :) Z(:, c), rows r0 .. n-1
    for (int i = r0 + tid; i < n; i += kT) {
      double v[W];
      const double* vr = V + (size_t)(i - r0) * ldv;
#pragma unroll
      for (int k = 0; k < W; ++k) v[k] = k < w ? __ldcg(vr + k) : 0.0;
      double* base = a.H + i;
      for (int q = 0; q < nc; ++q) {
        double* px = base + (size_t)(cc + q) * n;
        double x = __ldcg(px);
#pragma unroll
        for (int k = 0; k < W; ++k) x = fma(-v[k], Zs[k * kSCmax + q], x);
        *px = x;
      }
    }
  }
  __syncthreads();
}

// Phase C, top part: right update A_ext(i, c) -= Y(i, :) V(c - r0, :)^T of the
// rows above r0 and of C (extended row t < r0 ? t : n + t - r0, t < r0 + p)
// and the columns r0 .. n-1, as kTR x kTC tiles with Y and V staged in shared
// memory (so the tile runs at full width however few rows there are).
template <int W>
__device__ void top_tile(const RedArgs& a, int r0, int w, const double* __restrict__ V, int ldv,
                         int tile, double* sm) {
  const int n = a.n, rt = r0 + a.p;
  const int ntc = (n - r0 + kTC - 1) / kTC;
  const int t0 = (tile / ntc) * kTR, c0 = r0 + (tile % ntc) * kTC;
  const int R = min(kTR, rt - t0), C = min(kTC, n - c0);
  double* Yt = sm;
  double* Vt = Yt + kTR * kVLD;
  const int tid = threadIdx.x;
  __syncthreads();
  for (int e = tid; e < R * W; e += kT) {
    const int r = e / W, k = e % W;
    const int t = t0 + r;
    const int i = t < r0 ? t : n + (t - r0);
    Yt[r * kVLD + k] = __ldcg(a.Y + (size_t)i * kW + k);
  }
  for (int e = tid; e < C * W; e += kT) {
    const int q = e / W, k = e % W;
    Vt[q * kVLD + k] = k < w ? __ldcg(V + (size_t)(c0 + q - r0) * ldv + k) : 0.0;
  }
  __syncthreads();
  for (int e = tid; e < R * C; e += kT) {
    const int r = e % R, q = e / R;
    const int t = t0 + r;
    const int i = t < r0 ? t : n + (t - r0);
    size_t ld = 0;
    double* px = ext_row(a, i, &ld) + (size_t)(c0 + q) * ld;
    double x = __ldcg(px);
    const double* yr = Yt + r * kVLD;
    const double* vq = Vt + q * kVLD;
#pragma unroll
    for (int k = 0; k < W; ++k) x = fma(-yr[k], vq[k], x);
    *px = x;
  }
}

template <int W>
__device__ void block_step(const RedArgs& a, int r0, int lc, int w, const double* V, int ldv,
                           const double* Ts, int wn, int tn, double* work, bool* ok) {
  const int n = a.n, m = a.m, p = a.p;
  phase_b<W>(a, r0, w, V, ldv, Ts, work);
  if (!grid_barrier(a.bar, a.err, kBarrierSpins)) { *ok = false; return; }
  if (blockIdx.x == 0) {
    // look-ahead: the next panel's columns (rows r0 .. n-1), then its QR
    if (wn > 0) {
      phase_c_bottom<W>(a, r0, w, V, ldv, Ts, lc, lc + wn, work);
      const int rn = lc + m;
      panel_qr(a.H + rn + (size_t)lc * n, (size_t)n, n - rn, wn, wn, wn, a.tauA + lc,
               a.VA + (size_t)(tn & 1) * n * kW, kW, a.TA + (size_t)(tn & 1) * kSmT, work);
    }
  } else {
    // the other blocks split, by multiply-add count, the bottom columns
    // [lc + wn, n) (3 (n - r0) w each) followed by the top tiles
    // (kTR kTC w each; plus a fixed charge for the staging of a tile)
    const long long nB = n - lc - wn;
    const int rt = r0 + p;
    const long long nT = rt > 0 ? (long long)((rt + kTR - 1) / kTR) * ((n - r0 + kTC - 1) / kTC) : 0;
    const long long cB = 3LL * (n - r0) * w + 64;
    const long long cT = (long long)kTR * kTC * w + 2048;
    const long long tot = nB * cB + nT * cT;
    const int G = gridDim.x - 1, b = blockIdx.x - 1;
    const long long lo = tot * b / G, hi = tot * (b + 1) / G;
    auto first = [](long long x, long long c, long long cnt) -> long long {
      if (x <= 0) return 0;
      const long long k = (x + c - 1) / c;
      return k < cnt ? k : cnt;
    };
    const int bb0 = (int)first(lo, cB, nB), bb1 = (int)first(hi, cB, nB);
    if (bb1 > bb0) phase_c_bottom<W>(a, r0, w, V, ldv, Ts, lc + wn + bb0, lc + wn + bb1, work);
    if (nT > 0) {
      const int tt0 = (int)first(lo - nB * cB, cT, nT), tt1 = (int)first(hi - nB * cB, cT, nT);
      for (int tile = tt0; tile < tt1; ++tile) top_tile<W>(a, r0, w, V, ldv, tile, work);
    }
  }
  if (!grid_barrier(a.bar, a.err, kBarrierSpins)) *ok = false;
}

__global__ void __launch_bounds__(kT, 1) reduce_blocked_kernel(RedArgs a) {
  extern __shared__ double sm[];
  double* Ts = sm;              // T of the current step
  double* work = sm + kSmT;
  const int n = a.n, m = a.m;
  // Step 1 of Algorithm 1: QR of B (block 0), reflectors grouped by kW
  if (blockIdx.x == 0 && a.kb > 0)
    panel_qr(a.R, (size_t)n, n, a.kb, m, kW, a.tauB, a.VB, a.kb, a.TB, work);
  const int nbB = (a.kb + kW - 1) / kW;
  const int naA = a.ka > 0 ? (a.ka + a.wa - 1) / a.wa : 0;
  const int nsteps = nbB + naA;
  // the first A panel, when there is no B step to look ahead from
  if (nbB == 0 && naA > 0 && blockIdx.x == 0) {
    const int w1 = min(a.wa, a.ka);
    panel_qr(a.H + m, (size_t)n, n - m, w1, w1, w1, a.tauA, a.VA, kW, a.TA, work);
  }
  if (!grid_barrier(a.bar, a.err, kBarrierSpins)) return;
  for (int s = 0; s < nsteps; ++s) {
    int r0, lc, w, ldv;
    const double* V;
    const double* T;
    if (s < nbB) {
      const int q0 = s * kW;
      w = min(kW, a.kb - q0);
      r0 = q0;
      lc = 0;
      V = a.VB + (size_t)q0 * a.kb + q0;
      ldv = a.kb;
      T = a.TB + (size_t)s * kSmT;
    } else {
      const int t = s - nbB;
      const int j0 = t * a.wa;
      w = min(a.wa, a.ka - j0);
      r0 = j0 + m;
      lc = j0 + w;
      V = a.VA + (size_t)(t & 1) * n * kW;
      ldv = kW;
      T = a.TA + (size_t)(t & 1) * kSmT;
    }
    for (int e = threadIdx.x; e < kSmT; e += kT) Ts[e] = __ldcg(T + e);
    __syncthreads();
    // the next step's panel (an A mini-block) starts at column lc
    const bool next_a = s + 1 < nsteps && s + 1 >= nbB;
    const int tn = s + 1 - nbB;
    const int wn = next_a ? min(a.wa, a.ka - tn * a.wa) : 0;
    bool ok = true;
    if (w <= 1) block_step<1>(a, r0, lc, w, V, ldv, Ts, wn, tn, work, &ok);
    else if (w <= 2) block_step<2>(a, r0, lc, w, V, ldv, Ts, wn, tn, work, &ok);
    else if (w <= 4) block_step<4>(a, r0, lc, w, V, ldv, Ts, wn, tn, work, &ok);
    else block_step<8>(a, r0, lc, w, V, ldv, Ts, wn, tn, work, &ok);
    if (!ok) return;
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
  if (h->kb <= 0 && h->ka <= 0) return SSV_OK;
  const int kb = std::max(h->kb, 0);
  const int nbB = (kb + kW - 1) / kW;
  const size_t ndbl = (size_t)n * kb + (size_t)nbB * kSmT + 2 * (size_t)n * kW + 2 * (size_t)kSmT +
                      (size_t)np * kW;
  const size_t bytes = sizeof(double) * ndbl + 4 * sizeof(unsigned) + 16;
  unsigned char* wsp = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&wsp, bytes, st));
  RedArgs a;
  a.H = h->H; a.R = h->R; a.Ct = h->Ct; a.tauA = h->tauA; a.tauB = h->tauB;
  a.n = n; a.m = m; a.p = p; a.ldct = p > 0 ? p : 1; a.kb = kb; a.ka = h->ka;
  a.wa = std::min(m, kWA);
  double* d = reinterpret_cast<double*>(wsp);
  a.VB = d;
  a.TB = a.VB + (size_t)n * kb;
  a.VA = a.TB + (size_t)nbB * kSmT;
  a.TA = a.VA + 2 * (size_t)n * kW;
  a.Y = a.TA + 2 * (size_t)kSmT;
  a.bar = reinterpret_cast<unsigned*>(d + ndbl);
  a.err = reinterpret_cast<int*>(a.bar + 2);
  int rc = SSV_OK;
  cudaError_t e = cudaMemsetAsync(a.bar, 0, 4 * sizeof(unsigned), st);
  const size_t smem = sizeof(double) * kSmDoubles;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(reduce_blocked_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
  int occ = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, reduce_blocked_kernel, kT, smem);
  if (e == cudaSuccess && occ < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) {
    const int grid = std::max(2, num_sms());
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel((const void*)reduce_blocked_kernel, dim3(grid), dim3(kT), args,
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
  SSV_CUDA_TRY(pool_alloc((void**)&wsp, 16, st));
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
