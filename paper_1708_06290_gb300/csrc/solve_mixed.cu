// Mixed-precision shifted solve: complex64 elimination sweeps with iterative
// refinement whose residual R - (H - sigma I) Xhat is computed FP64-accurately.
//
// Per shift, one thread block runs
//   1. sweep 0: the blocked bottom-up window elimination of Sec. 3.1 /
//      Algorithm 8 in complex64 (one Householder reflector per row over the m
//      live + 1 fresh candidate columns), carrying the rows of the accumulated
//      column transformation T (the "Q*" rows of Sec. 3.4), so that
//      Xhat0 = T(:, live) Wm^{-1} R(1:m, 1:m) is formed (stored in complex128);
//   2. refinement: E = R - (H - sigma I) Xhat with H = Hhi + Hlo (two FP32
//      words) and Xhat split the same way, each product formed exactly by an
//      FMA and accumulated in double-float (Dekker/Knuth two-sum), giving
//      ~48-bit residuals at FP32 throughput (native FP64 is 60x slower on
//      this GPU); the normwise backward error decides convergence;
//   3. a correction sweep solves (H - sigma I) D = E for the dense right-hand
//      side E by carrying E as extra window columns that are back-substituted
//      on the fly with each finalised column (the technique of Sec. 3.4 for
//      unreduced right-hand sides, here in the bottom-up RQ direction), and
//      Xhat += D.
// Shifts that do not reach the tolerance are flagged; the host re-solves them
// with the FP64 kernel.  Outputs: G = Ct Xhat (FP64) or Xhat.
#include <algorithm>

#include "ssv_internal.cuh"

namespace ssv {

namespace {

struct cf {
  float x, y;
};
__device__ __forceinline__ cf mkcf(float a, float b) { return cf{a, b}; }
__device__ __forceinline__ cf csubf(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
// a + b * c
__device__ __forceinline__ cf cfmaf(cf b, cf c, cf a) {
  return cf{fmaf(b.x, c.x, fmaf(-b.y, c.y, a.x)), fmaf(b.x, c.y, fmaf(b.y, c.x, a.y))};
}
// a - b * c
__device__ __forceinline__ cf cfmsf(cf b, cf c, cf a) {
  return cf{fmaf(-b.x, c.x, fmaf(b.y, c.y, a.x)), fmaf(-b.x, c.y, fmaf(-b.y, c.x, a.y))};
}
__device__ __forceinline__ float cabs1f(cf a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ cf cdivf(cf a, cf b) {
  if (fabsf(b.y) <= fabsf(b.x)) {
    float r = b.y / b.x, d = b.x + b.y * r;
    return cf{(a.x + a.y * r) / d, (a.y - a.x * r) / d};
  } else {
    float r = b.x / b.y, d = b.y + b.x * r;
    return cf{(a.x * r + a.y) / d, (a.y * r - a.x) / d};
  }
}

constexpr int kThreads = 256;
constexpr int kNB = 64;
constexpr int kJT = 32;  // residual: rows of Xhat staged per tile

template <int MAXM>
struct LayoutM {
  static constexpr int S = MAXM + 2;       // m live + two alternating fresh slots
  static constexpr int CR = kNB + MAXM;    // coefficient rows: fresh, then old live
  static constexpr size_t cand = (size_t)S * kNB;
  static constexpr size_t rhs = (size_t)MAXM * kNB;
  static constexpr size_t coef = (size_t)CR * S;
  static constexpr size_t coefr = (size_t)CR * MAXM;
  static constexpr size_t vref = MAXM + 4;
  static constexpr size_t wm = (size_t)MAXM * 2 * MAXM;
  static constexpr size_t yb = (size_t)MAXM * MAXM;
  static constexpr size_t cf_elems = cand + rhs + coef + coefr + vref + wm + yb;
  static constexpr size_t xs_floats = (size_t)kJT * MAXM * 4;
  static constexpr size_t bytes =
      ((cf_elems * sizeof(cf) + 15) / 16) * 16 + xs_floats * sizeof(float) + 64 * sizeof(double);
};

template <int MAXM>
struct Smem {
  cf* cand;
  cf* rhs;
  cf* coef;
  cf* coefr;
  cf* vref;
  cf* wm;
  cf* yb;
  float4* xs;
  double* red;
  __device__ void bind(unsigned char* raw) {
    using L = LayoutM<MAXM>;
    cand = reinterpret_cast<cf*>(raw);
    rhs = cand + L::cand;
    coef = rhs + L::rhs;
    coefr = coef + L::coef;
    vref = coefr + L::coefr;
    wm = vref + L::vref;
    yb = wm + L::wm;
    xs = reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(raw) +
                                   ((L::cf_elems * sizeof(cf) + 15) / 16) * 16);
    red = reinterpret_cast<double*>(reinterpret_cast<unsigned char*>(xs) + L::xs_floats * sizeof(float));
  }
};

// s = s_hi + s_lo accumulates a_hi*b_hi exactly (FMA error term) plus the FP32
// cross terms a_hi*b_lo + a_lo*b_hi; the high sum is kept with two-sum.
__device__ __forceinline__ void df_mac(float& s_hi, float& s_lo, float a_hi, float a_lo, float b_hi,
                                       float b_lo) {
  const float p = a_hi * b_hi;
  const float e = fmaf(a_hi, b_hi, -p);
  const float t = fmaf(a_hi, b_lo, fmaf(a_lo, b_hi, e));
  const float s = s_hi + p;
  const float bp = s - s_hi;
  const float err = (s_hi - (s - bp)) + (p - bp);
  s_hi = s;
  s_lo += err + t;
}

// Block-wide sum of two doubles; every thread gets the totals.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[w] = a;
    red[32 + w] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
  for (int i = 0; i < nw; ++i) {
    a += red[i];
    b += red[32 + i];
  }
  __syncthreads();
}

// One complex64 elimination sweep over H - sigma I (rows n-1 .. m).
// Live columns Zl (n x m), their T rows Tl (n x m).  With RHS, the dense
// right-hand side Zr (n x m) is back-substituted on the fly and its T rows
// accumulate in Tr.  On return Zl(0:m, :) = Wm, Zr(0:m, :) = remaining RHS.
// Returns (through sm.red[63]) 1 if a finalised diagonal fell below sing_tol.
template <int MAXM, bool RHS>
__device__ void sweep(const int n, const int m, const int nb, const float* __restrict__ Hhi,
                      const cf sigma, cf* __restrict__ Zl, cf* __restrict__ Zr,
                      cf* __restrict__ Tl, cf* __restrict__ Tr, Smem<MAXM>& sm,
                      const float sing_tol, int* s_flag) {
  constexpr int S = LayoutM<MAXM>::S;
  constexpr int CR = LayoutM<MAXM>::CR;
  const int tid = threadIdx.x;
  // live columns: the last m columns of H - sigma I; T rows: unit vectors
  for (long long idx = tid; idx < (long long)n * m; idx += kThreads) {
    const int i = (int)(idx % n), q = (int)(idx / n);
    const int j = n - m + q;
    cf z = mkcf(Hhi[i + (size_t)j * n], 0.0f);
    if (i == j) z = csubf(z, sigma);
    Zl[idx] = z;
    Tl[idx] = mkcf(i == j ? 1.0f : 0.0f, 0.0f);
    if (RHS) Tr[idx] = mkcf(0.0f, 0.0f);
  }
  __syncthreads();
  int k = n;
  while (k > m) {
    const int nbe = min(nb, k - m);
    const int r = k - nbe;
    const int j0 = k - m - nbe;
    for (int idx = tid; idx < m * nbe; idx += kThreads) {
      const int t = idx % nbe, q = idx / nbe;
      sm.cand[q * kNB + t] = Zl[(r + t) + (size_t)q * n];
      if (RHS) sm.rhs[q * kNB + t] = Zr[(r + t) + (size_t)q * n];
    }
    for (int idx = tid; idx < CR * S; idx += kThreads) {
      const int c = idx / S, slot = idx % S;
      float v = ((slot < m && c == kNB + slot) || (slot == m && c == nbe - 1)) ? 1.0f : 0.0f;
      sm.coef[idx] = mkcf(v, 0.0f);
    }
    if (RHS)
      for (int idx = tid; idx < CR * MAXM; idx += kThreads) sm.coefr[idx] = mkcf(0.0f, 0.0f);
    {
      const int c = nbe - 1, jc = j0 + c;
      for (int t = tid; t <= c; t += kThreads) {
        cf z = mkcf(Hhi[(r + t) + (size_t)jc * n], 0.0f);
        if (t == c - m) z = csubf(z, sigma);
        sm.cand[m * kNB + t] = z;
      }
    }
    __syncthreads();
    for (int c = nbe - 1; c >= 0; --c) {
      const int fs = m + ((nbe - 1 - c) & 1);
      const int fn = (fs == m) ? m + 1 : m;
      if (tid < 32) {
        float rest2 = 0.0f;
        for (int q = tid; q < m; q += 32) {
          const cf x = sm.cand[q * kNB + c];
          rest2 = fmaf(x.x, x.x, fmaf(x.y, x.y, rest2));
        }
        for (int o = 16; o > 0; o >>= 1) rest2 += __shfl_xor_sync(0xffffffffu, rest2, o);
        const cf xf = sm.cand[fs * kNB + c];
        const float af2 = fmaf(xf.x, xf.x, xf.y * xf.y);
        const float af = sqrtf(af2);
        const float nrm2 = rest2 + af2;
        const float nrm = sqrtf(nrm2);
        const cf ph = af > 0.0f ? mkcf(xf.x / af, -xf.y / af) : mkcf(1.0f, 0.0f);
        const cf alpha = mkcf(-ph.x * nrm, -ph.y * nrm);
        const bool trivial = !(rest2 > 0.0f);
        for (int q = tid; q <= m; q += 32) {
          const int slot = q < m ? q : fs;
          const cf x = sm.cand[slot * kNB + c];
          cf v = mkcf(x.x, -x.y);
          if (slot == fs) v = csubf(v, alpha);
          sm.vref[slot] = v;
        }
        if (tid == 0) {
          const float vv = 2.0f * nrm2 + 2.0f * af * nrm;
          sm.vref[MAXM + 2].x = trivial ? 0.0f : 2.0f / vv;
          // finalised diagonal entry: conj(alpha) (or x_fs when no reflection)
          sm.vref[MAXM + 3] = trivial ? xf : mkcf(alpha.x, -alpha.y);
          if (nrm <= sing_tol) *s_flag = 1;
        }
      }
      __syncthreads();
      const float tau = sm.vref[MAXM + 2].x;
      if (tau != 0.0f) {
        const int nrow = c;
        const int ncoef = (nbe - c) + m;
        for (int e = tid; e < nrow + ncoef; e += kThreads) {
          cf* base;
          int stride;
          if (e < nrow) {
            base = sm.cand + e;
            stride = kNB;
          } else {
            const int ee = e - nrow;
            const int crow = ee < nbe - c ? c + ee : kNB + (ee - (nbe - c));
            base = sm.coef + crow * S;
            stride = 1;
          }
          cf w = mkcf(0.0f, 0.0f);
          for (int q = 0; q <= m; ++q) {
            const int slot = q < m ? q : fs;
            w = cfmaf(base[slot * stride], sm.vref[slot], w);
          }
          w = mkcf(w.x * tau, w.y * tau);
          for (int q = 0; q <= m; ++q) {
            const int slot = q < m ? q : fs;
            const cf vc = mkcf(sm.vref[slot].x, -sm.vref[slot].y);
            base[slot * stride] = cfmsf(w, vc, base[slot * stride]);
          }
        }
      }
      if (RHS) {
        __syncthreads();
        // back substitution with the finalised column (slot fs): the RHS
        // entries of row c vanish, rows above and coefficients follow.
        const cf beta = sm.vref[MAXM + 3];
        const int nrow = c;
        const int ncoef = (nbe - c) + m;
        for (int idx = tid; idx < (nrow + ncoef) * m; idx += kThreads) {
          const int e = idx / m, q = idx % m;
          const cf f = (beta.x == 0.0f && beta.y == 0.0f) ? mkcf(0.0f, 0.0f)
                                                          : cdivf(sm.rhs[q * kNB + c], beta);
          if (e < nrow) {
            sm.rhs[q * kNB + e] = cfmsf(f, sm.cand[fs * kNB + e], sm.rhs[q * kNB + e]);
          } else {
            const int ee = e - nrow;
            const int crow = ee < nbe - c ? c + ee : kNB + (ee - (nbe - c));
            sm.coefr[crow * MAXM + q] = cfmsf(f, sm.coef[crow * S + fs], sm.coefr[crow * MAXM + q]);
          }
        }
      }
      if (c > 0) {
        const int cn = c - 1, jc = j0 + cn;
        for (int t = tid; t <= cn; t += kThreads) {
          cf z = mkcf(Hhi[(r + t) + (size_t)jc * n], 0.0f);
          if (t == cn - m) z = csubf(z, sigma);
          sm.cand[fn * kNB + t] = z;
        }
        for (int crow = tid; crow < CR; crow += kThreads)
          sm.coef[crow * S + fn] = mkcf(crow == cn ? 1.0f : 0.0f, 0.0f);
      }
      __syncthreads();
    }

    // ---- rows above the block
    for (int i = tid; i < r; i += kThreads) {
      cf al[MAXM];
      cf ar[RHS ? MAXM : 1];
#pragma unroll
      for (int q = 0; q < MAXM; ++q) al[q] = mkcf(0.0f, 0.0f);
      if (RHS) {
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) ar[q] = Zr[i + (size_t)q * n];
      }
      for (int c = 0; c < nbe; ++c) {
        const float z = Hhi[i + (size_t)(j0 + c) * n];
        const cf* cr = sm.coef + c * S;
#pragma unroll
        for (int q = 0; q < MAXM; ++q) {
          if (q < m) {
            al[q].x = fmaf(z, cr[q].x, al[q].x);
            al[q].y = fmaf(z, cr[q].y, al[q].y);
          }
        }
        if (RHS) {
          const cf* rr = sm.coefr + c * MAXM;
#pragma unroll
          for (int q = 0; q < MAXM; ++q) {
            if (q < m) {
              ar[q].x = fmaf(z, rr[q].x, ar[q].x);
              ar[q].y = fmaf(z, rr[q].y, ar[q].y);
            }
          }
        }
      }
      for (int qq = 0; qq < m; ++qq) {
        const cf zz = Zl[i + (size_t)qq * n];
        const cf* cr = sm.coef + (kNB + qq) * S;
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) al[q] = cfmaf(zz, cr[q], al[q]);
        if (RHS) {
          const cf* rr = sm.coefr + (kNB + qq) * MAXM;
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            if (q < m) ar[q] = cfmaf(zz, rr[q], ar[q]);
        }
      }
      const int cd_ = i - (r - m);
      if (cd_ >= 0 && cd_ < min(m, nbe)) {
        const cf* cr = sm.coef + cd_ * S;
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) al[q] = cfmsf(sigma, cr[q], al[q]);
        if (RHS) {
          const cf* rr = sm.coefr + cd_ * MAXM;
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            if (q < m) ar[q] = cfmsf(sigma, rr[q], ar[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < MAXM; ++q) {
        if (q < m) {
          Zl[i + (size_t)q * n] = al[q];
          if (RHS) Zr[i + (size_t)q * n] = ar[q];
        }
      }
    }
    // ---- T rows j0 .. n-1
    {
      const int lo = k - m;
      for (int i = j0 + tid; i < n; i += kThreads) {
        cf al[MAXM];
        cf ar[RHS ? MAXM : 1];
        if (i < lo) {
#pragma unroll
          for (int q = 0; q < MAXM; ++q) al[q] = sm.coef[(i - j0) * S + q];
          if (RHS) {
#pragma unroll
            for (int q = 0; q < MAXM; ++q) ar[q] = sm.coefr[(i - j0) * MAXM + q];
          }
        } else {
#pragma unroll
          for (int q = 0; q < MAXM; ++q) al[q] = mkcf(0.0f, 0.0f);
          if (RHS) {
#pragma unroll
            for (int q = 0; q < MAXM; ++q)
              if (q < m) ar[q] = Tr[i + (size_t)q * n];
          }
          for (int qq = 0; qq < m; ++qq) {
            const cf tt = Tl[i + (size_t)qq * n];
            const cf* cr = sm.coef + (kNB + qq) * S;
#pragma unroll
            for (int q = 0; q < MAXM; ++q)
              if (q < m) al[q] = cfmaf(tt, cr[q], al[q]);
            if (RHS) {
              const cf* rr = sm.coefr + (kNB + qq) * MAXM;
#pragma unroll
              for (int q = 0; q < MAXM; ++q)
                if (q < m) ar[q] = cfmaf(tt, rr[q], ar[q]);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < MAXM; ++q) {
          if (q < m) {
            Tl[i + (size_t)q * n] = al[q];
            if (RHS) Tr[i + (size_t)q * n] = ar[q];
          }
        }
      }
    }
    __syncthreads();
    k -= nbe;
  }
}

// Solve Wm Y = B (m x m, complex64) by Gauss-Jordan with partial pivoting;
// Wm = Zl(0:m, :); B = R(0:m, 0:m) (RHS == false) or Zr(0:m, :) (RHS == true).
template <int MAXM, bool RHS>
__device__ void final_solve(const int n, const int m, const cf* Zl, const cf* Zr,
                            const double* __restrict__ R, Smem<MAXM>& sm, const float sing_tol,
                            int* s_flag, int* s_piv) {
  const int tid = threadIdx.x;
  cf* W = sm.wm;
  const int w2 = 2 * m;
  for (int idx = tid; idx < m * w2; idx += kThreads) {
    const int i = idx % m, j = idx / m;
    cf v;
    if (j < m) v = Zl[i + (size_t)j * n];
    else if (RHS) v = Zr[i + (size_t)(j - m) * n];
    else v = mkcf(i <= j - m ? (float)R[i + (size_t)(j - m) * n] : 0.0f, 0.0f);
    W[i + j * MAXM] = v;
  }
  __syncthreads();
  for (int kk = 0; kk < m; ++kk) {
    if (tid < 32) {
      float best = -1.0f;
      int brow = kk;
      for (int i = kk + tid; i < m; i += 32) {
        const float v = cabs1f(W[i + kk * MAXM]);
        if (v > best) { best = v; brow = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
        if (ob > best || (ob == best && orow < brow)) { best = ob; brow = orow; }
      }
      if (tid == 0) {
        *s_piv = brow;
        const cf pv = W[brow + kk * MAXM];
        if (best == 0.0f || sqrtf(pv.x * pv.x + pv.y * pv.y) <= sing_tol) *s_flag = 1;
      }
    }
    __syncthreads();
    const int pr = *s_piv;
    if (pr != kk) {
      for (int j = tid; j < w2; j += kThreads) {
        const cf a = W[kk + j * MAXM];
        W[kk + j * MAXM] = W[pr + j * MAXM];
        W[pr + j * MAXM] = a;
      }
    }
    __syncthreads();
    const cf d = W[kk + kk * MAXM];
    const bool dz = (d.x == 0.0f && d.y == 0.0f);
    if (tid < m) sm.vref[tid] = (tid == kk || dz) ? mkcf(0.0f, 0.0f) : cdivf(W[tid + kk * MAXM], d);
    __syncthreads();
    for (int idx = tid; idx < m * w2; idx += kThreads) {
      const int i = idx % m, j = idx / m;
      if (i != kk && j > kk) W[i + j * MAXM] = cfmsf(sm.vref[i], W[kk + j * MAXM], W[i + j * MAXM]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * m; idx += kThreads) {
    const int i = idx % m, q = idx / m;
    const cf d = W[i + i * MAXM];
    sm.yb[i + q * MAXM] = (d.x == 0.0f && d.y == 0.0f) ? mkcf(0.0f, 0.0f) : cdivf(W[i + (m + q) * MAXM], d);
  }
  __syncthreads();
}

// E = R - (H - sigma I) Xhat, FP64-accurate; E rounded to complex64 into Zr.
// Returns ||E||_F^2 and ||Xhat||_F^2 (all threads).
template <int MAXM>
__device__ void residual(const int n, const int m, const float* __restrict__ Hhi,
                         const float* __restrict__ Hlo, const double* __restrict__ R,
                         const cd sigma, const cd* __restrict__ Xh, cf* __restrict__ Zr,
                         Smem<MAXM>& sm, double& e2, double& x2) {
  const int tid = threadIdx.x;
  e2 = 0.0;
  x2 = 0.0;
  for (int i0 = 0; i0 < n; i0 += kThreads) {
    const int i = i0 + tid;
    float rh[MAXM], rl[MAXM], ih[MAXM], il[MAXM];
#pragma unroll
    for (int q = 0; q < MAXM; ++q) { rh[q] = 0.f; rl[q] = 0.f; ih[q] = 0.f; il[q] = 0.f; }
    const int jlo = max(0, i0 - m);
    for (int jt = jlo; jt < n; jt += kJT) {
      __syncthreads();
      for (int idx = tid; idx < kJT * m; idx += kThreads) {
        const int jj = idx % kJT, q = idx / kJT;
        const int j = jt + jj;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n) {
          const cd x = Xh[j + (size_t)q * n];
          const float a = (float)x.x, b = (float)x.y;
          v = make_float4(a, (float)(x.x - (double)a), b, (float)(x.y - (double)b));
        }
        sm.xs[jj * MAXM + q] = v;
      }
      __syncthreads();
      if (i < n) {
        const int jend = min(kJT, n - jt);
        for (int jj = 0; jj < jend; ++jj) {
          const int j = jt + jj;
          float hh = 0.f, hl = 0.f;
          if (j >= i - m) {
            hh = Hhi[i + (size_t)j * n];
            hl = Hlo[i + (size_t)j * n];
          }
#pragma unroll
          for (int q = 0; q < MAXM; ++q) {
            if (q < m) {
              const float4 x = sm.xs[jj * MAXM + q];
              df_mac(rh[q], rl[q], hh, hl, x.x, x.y);
              df_mac(ih[q], il[q], hh, hl, x.z, x.w);
            }
          }
        }
      }
    }
    if (i < n) {
#pragma unroll
      for (int q = 0; q < MAXM; ++q) {
        if (q < m) {
          const cd x = Xh[i + (size_t)q * n];
          const double hxr = (double)rh[q] + (double)rl[q];
          const double hxi = (double)ih[q] + (double)il[q];
          // E = R - H x + sigma x
          double er = -hxr + (sigma.x * x.x - sigma.y * x.y);
          double ei = -hxi + (sigma.x * x.y + sigma.y * x.x);
          if (i <= q) er += R[i + (size_t)q * n];
          e2 += er * er + ei * ei;
          x2 += x.x * x.x + x.y * x.y;
          Zr[i + (size_t)q * n] = mkcf((float)er, (float)ei);
        }
      }
    }
  }
  block_sum2(e2, x2, sm.red);
}

template <int MAXM>
__global__ void __launch_bounds__(kThreads) solve_mixed_kernel(
    int n, int m, int p, int nb, const float* __restrict__ Hhi, const float* __restrict__ Hlo,
    const double* __restrict__ R, const double* __restrict__ Ct, int ldct, int s,
    const cd* __restrict__ shifts, int mode, unsigned char* __restrict__ scratch,
    size_t slot_bytes, cd* __restrict__ out, long long ldo, int* __restrict__ status,
    double* __restrict__ resid, int* __restrict__ fallback, const double* __restrict__ hnorm,
    int max_refine, double tol) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<MAXM> sm;
  sm.bind(smem_raw);
  __shared__ int s_flag;
  __shared__ int s_piv;
  const int tid = threadIdx.x;
  unsigned char* base = scratch + (size_t)blockIdx.x * slot_bytes;
  const size_t nm = (size_t)n * m;
  cd* Xh = reinterpret_cast<cd*>(base);
  cf* Zl = reinterpret_cast<cf*>(base + nm * sizeof(cd));
  cf* Zr = Zl + nm;
  cf* Tl = Zr + nm;
  cf* Tr = Tl + nm;

  double r2 = 0.0;  // ||R(0:m,0:m)||_F^2
  for (int q = 0; q < m; ++q)
    for (int i = 0; i <= q; ++i) r2 += R[i + (size_t)q * n] * R[i + (size_t)q * n];
  const double rnorm = sqrt(r2);

  for (int sh = blockIdx.x; sh < s; sh += gridDim.x) {
    const cd sigma = shifts[sh];
    const cf sigf = mkcf((float)sigma.x, (float)sigma.y);
    const double mnorm = sqrt(fmax(hnorm[0] - 2.0 * sigma.x * hnorm[1] +
                                       (double)n * (sigma.x * sigma.x + sigma.y * sigma.y), 0.0));
    const float sing_tol = (float)((double)n * 1.1920928955078125e-07 * mnorm);
    if (tid == 0) s_flag = 0;
    __syncthreads();
    // ---- sweep 0 -> Xhat0
    sweep<MAXM, false>(n, m, nb, Hhi, sigf, Zl, Zr, Tl, Tr, sm, sing_tol, &s_flag);
    final_solve<MAXM, false>(n, m, Zl, Zr, R, sm, sing_tol, &s_flag, &s_piv);
    for (long long idx = tid; idx < (long long)nm; idx += kThreads) {
      const int i = (int)(idx % n), q = (int)(idx / n);
      float ar = 0.f, ai = 0.f;
      for (int t = 0; t < m; ++t) {
        const cf a = Tl[i + (size_t)t * n];
        const cf y = sm.yb[t + q * MAXM];
        ar = fmaf(a.x, y.x, fmaf(-a.y, y.y, ar));
        ai = fmaf(a.x, y.y, fmaf(a.y, y.x, ai));
      }
      Xh[idx] = mkcd(ar, ai);
    }
    __syncthreads();
    // ---- refinement
    double eta = INFINITY, eta_prev = INFINITY;
    bool ok = false;
    for (int it = 0;; ++it) {
      double e2, x2;
      residual<MAXM>(n, m, Hhi, Hlo, R, sigma, Xh, Zr, sm, e2, x2);
      eta = sqrt(e2) / (mnorm * sqrt(x2) + rnorm);
      if (!(eta == eta)) break;  // NaN
      if (eta <= tol) { ok = true; break; }
      if (it >= max_refine || eta > 0.5 * eta_prev || s_flag) break;
      eta_prev = eta;
      sweep<MAXM, true>(n, m, nb, Hhi, sigf, Zl, Zr, Tl, Tr, sm, sing_tol, &s_flag);
      final_solve<MAXM, true>(n, m, Zl, Zr, R, sm, sing_tol, &s_flag, &s_piv);
      // Xhat += Tl Y - Tr
      for (long long idx = tid; idx < (long long)nm; idx += kThreads) {
        const int i = (int)(idx % n), q = (int)(idx / n);
        const cf tr = Tr[idx];
        float ar = -tr.x, ai = -tr.y;
        for (int t = 0; t < m; ++t) {
          const cf a = Tl[i + (size_t)t * n];
          const cf y = sm.yb[t + q * MAXM];
          ar = fmaf(a.x, y.x, fmaf(-a.y, y.y, ar));
          ai = fmaf(a.x, y.y, fmaf(a.y, y.x, ai));
        }
        cd x = Xh[idx];
        x.x += (double)ar;
        x.y += (double)ai;
        Xh[idx] = x;
      }
      __syncthreads();
    }
    // ---- outputs
    if (ok) {
      if (mode == SSV_G || mode == SSV_TF) {
        const double sg = mode == SSV_TF ? -1.0 : 1.0;
        cd* o = out + (size_t)sh * m * ldo;
        for (int idx = tid; idx < p * m; idx += kThreads) {
          const int i = idx % p, q = idx / p;
          double ar = 0.0, ai = 0.0;
          for (int t = 0; t < n; ++t) {
            const double c = Ct[i + (size_t)t * ldct];
            const cd x = Xh[t + (size_t)q * n];
            ar = fma(c, x.x, ar);
            ai = fma(c, x.y, ai);
          }
          o[i + (size_t)q * ldo] = mkcd(sg * ar, sg * ai);
        }
      } else {
        cd* o = out + (size_t)sh * m * ldo;
        for (long long idx = tid; idx < (long long)nm; idx += kThreads) {
          const int i = (int)(idx % n), q = (int)(idx / n);
          o[i + (size_t)q * ldo] = Xh[idx];
        }
      }
    }
    if (tid == 0) {
      if (status) status[sh] = ok ? SSV_SHIFT_OK : SSV_SHIFT_NOT_CONVERGED;
      if (resid) resid[sh] = eta;
      fallback[sh] = ok ? 0 : 1;
    }
    __syncthreads();
  }
}

template <int MAXM>
int launch_mixed(const Handle* h, int s, const double* shifts, int nb, int mode, double* out,
                 long long ldo, int* status, double* resid, int* fallback, int max_refine,
                 double tol, cudaStream_t st) {
  using L = LayoutM<MAXM>;
  const int n = h->n, m = h->m, p = h->p;
  const size_t slot = (size_t)n * m * (sizeof(cd) + 4 * sizeof(cf));
  auto kern = solve_mixed_kernel<MAXM>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
  int per_sm = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L::bytes));
  per_sm = std::max(1, std::min(per_sm, 4));
  const int grid = std::min(s, num_sms() * per_sm);
  unsigned char* scratch = nullptr;
  SSV_CUDA_TRY(cudaMallocAsync((void**)&scratch, slot * grid, st));
  kern<<<grid, kThreads, L::bytes, st>>>(n, m, p, nb, h->Hhi, h->Hlo, h->R, h->Ct, p > 0 ? p : 1, s,
                                         reinterpret_cast<const cd*>(shifts), mode, scratch, slot,
                                         reinterpret_cast<cd*>(out), ldo, status, resid, fallback,
                                         h->hnorm2, max_refine, tol);
  count_launch();
  cudaError_t e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return SSV_ECUDA;
  }
  return SSV_OK;
}

}  // namespace

size_t solve_mixed_scratch_bytes(int n, int m, int p, int s, const ssv_opts* o) {
  (void)p;
  (void)o;
  const size_t slot = (size_t)n * m * (sizeof(cd) + 4 * sizeof(cf));
  const size_t grid = (size_t)std::min(s, num_sms() * 4);
  return slot * grid + sizeof(int) * (size_t)s + 256;
}

int solve_mixed(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                long long ldo, int* status, double* resid, cudaStream_t st) {
  const int m = h->m;
  const int nb = o->nb > 0 ? o->nb : default_nb(h->n, m);
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  int* fallback = nullptr;
  SSV_CUDA_TRY(cudaMallocAsync((void**)&fallback, sizeof(int) * (size_t)s, st));
  int rc;
  const int mode = o->mode == SSV_X ? SSV_XHAT : o->mode;
  if (m <= 1) rc = launch_mixed<1>(h, s, shifts, nb, mode, out, ldo, status, resid, fallback, o->max_refine, o->tol, st);
  else if (m <= 2) rc = launch_mixed<2>(h, s, shifts, nb, mode, out, ldo, status, resid, fallback, o->max_refine, o->tol, st);
  else if (m <= 4) rc = launch_mixed<4>(h, s, shifts, nb, mode, out, ldo, status, resid, fallback, o->max_refine, o->tol, st);
  else if (m <= 8) rc = launch_mixed<8>(h, s, shifts, nb, mode, out, ldo, status, resid, fallback, o->max_refine, o->tol, st);
  else if (m <= 16) rc = launch_mixed<16>(h, s, shifts, nb, mode, out, ldo, status, resid, fallback, o->max_refine, o->tol, st);
  else if (m <= 32) rc = launch_mixed<32>(h, s, shifts, nb, mode, out, ldo, status, resid, fallback, o->max_refine, o->tol, st);
  else rc = SSV_ENOTSUP;
  // shifts that did not converge: FP64 sweep (status and output overwritten);
  // their backward errors come from the FP64 solution
  if (rc == SSV_OK && resid == nullptr)
    rc = solve_fp64_masked(h, s, shifts, mode, 0, out, ldo, status, fallback, nullptr, 0, st);
  if (rc == SSV_OK && resid != nullptr) {
    cd* xcopy = nullptr;
    const bool gm = (mode == SSV_G || mode == SSV_TF);
    if (gm) {
      cudaError_t e = cudaMallocAsync((void**)&xcopy, sizeof(cd) * (size_t)h->n * m * s, st);
      if (e != cudaSuccess) { set_cuda_error(e); rc = SSV_ENOMEM; }
    }
    if (rc == SSV_OK)
      rc = solve_fp64_masked(h, s, shifts, mode, 0, out, ldo, status, fallback, xcopy, h->n, st);
    if (rc == SSV_OK)
      rc = backward_error_fp64_masked(h, s, shifts, gm ? reinterpret_cast<const double*>(xcopy) : out,
                                      gm ? h->n : ldo, resid, fallback, st);
    if (xcopy) cudaFreeAsync(xcopy, st);
  }
  cudaError_t e = cudaFreeAsync(fallback, st);
  if (e != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e);
    rc = SSV_ECUDA;
  }
  return rc;
}

}  // namespace ssv
