// Mixed-precision shifted solve: a first solve with double-float bulk updates,
// then iterative refinement with complex64 correction sweeps whose residual
// R - (H - sigma I) Xhat is computed FP64-accurately.
//
// Per shift:
//   1. first solve: the sweep of Sec. 3.1 / Algorithm 8 with its panels and
//      bulk updates (the rows above each block) in double-float on the FP32
//      pipe (SSV_DFLOAT); Xhat0 comes from the stored block transforms by a
//      backward pass (the "Q*" rows of Sec. 3.3 without per-step updates);
//   2. refinement residual: E = R - (H - sigma I) Xhat to FP64 accuracy.  For
//      m <= 16 on the tensor cores (residual_tc.cu: error-free BF16 digit
//      splitting of H and Xhat, exact FP32 accumulation per level); for wider
//      m with H = Hhi + Hlo (two FP32 words) and Xhat split the same way, each
//      product formed exactly by an FMA and accumulated in double-float
//      (Dekker / Knuth two-sum).  The normwise backward error decides
//      convergence;
//   3. a correction sweep in complex64 solves (H - sigma I) D = E for the dense
//      right-hand side E by carrying E as extra window columns that are
//      back-substituted on the fly with each finalised column (the technique
//      of Sec. 3.3 for unreduced right-hand sides, here in the bottom-up RQ
//      direction), and Xhat += D.
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

// a0/a1 (rows ia, ib < r) += sum_c Hhi(row, j0 + c) * P(c, :), P rows of `ps`
// complex entries in shared memory (16-byte aligned rows when MAXM >= 2).
template <int MAXM>
__device__ __forceinline__ void rows_real_times(const float* __restrict__ Hhi, int n, int j0,
                                                int nbe, int ia, int ib, int r, const cf* P,
                                                int ps, cf* a0, cf* a1) {
  const bool va = ia < r, vb = ib < r;
  for (int c0 = 0; c0 < nbe; c0 += 4) {
    float za[4], zb[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      za[u] = (va && c < nbe) ? Hhi[ia + (size_t)(j0 + c) * n] : 0.f;
      zb[u] = (vb && c < nbe) ? Hhi[ib + (size_t)(j0 + c) * n] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      if (c >= nbe) break;
      const cf* pr = P + c * ps;
      if constexpr (MAXM >= 2) {
        const float4* p4 = reinterpret_cast<const float4*>(pr);
#pragma unroll
        for (int q2 = 0; q2 < MAXM / 2; ++q2) {
          const float4 w = p4[q2];
          a0[2 * q2].x = fmaf(za[u], w.x, a0[2 * q2].x);
          a0[2 * q2].y = fmaf(za[u], w.y, a0[2 * q2].y);
          a0[2 * q2 + 1].x = fmaf(za[u], w.z, a0[2 * q2 + 1].x);
          a0[2 * q2 + 1].y = fmaf(za[u], w.w, a0[2 * q2 + 1].y);
          a1[2 * q2].x = fmaf(zb[u], w.x, a1[2 * q2].x);
          a1[2 * q2].y = fmaf(zb[u], w.y, a1[2 * q2].y);
          a1[2 * q2 + 1].x = fmaf(zb[u], w.z, a1[2 * q2 + 1].x);
          a1[2 * q2 + 1].y = fmaf(zb[u], w.w, a1[2 * q2 + 1].y);
        }
      } else {
        const cf w = pr[0];
        a0[0].x = fmaf(za[u], w.x, a0[0].x);
        a0[0].y = fmaf(za[u], w.y, a0[0].y);
        a1[0].x = fmaf(zb[u], w.x, a1[0].x);
        a1[0].y = fmaf(zb[u], w.y, a1[0].y);
      }
    }
  }
}

// a0/a1 += sum_qq Z(row, qq) * P(qq, :) for complex Z (n x m, ld n), rows < lim.
template <int MAXM>
__device__ __forceinline__ void rows_complex_times(const cf* __restrict__ Z, int n, int m, int ia,
                                                   int ib, int lim, const cf* P, int ps, cf* a0,
                                                   cf* a1) {
  const bool va = ia < lim, vb = ib < lim;
  for (int qq = 0; qq < m; ++qq) {
    const cf za = va ? Z[ia + (size_t)qq * n] : mkcf(0.f, 0.f);
    const cf zb = vb ? Z[ib + (size_t)qq * n] : mkcf(0.f, 0.f);
    const cf* pr = P + qq * ps;
    if constexpr (MAXM >= 2) {
      const float4* p4 = reinterpret_cast<const float4*>(pr);
#pragma unroll
      for (int q2 = 0; q2 < MAXM / 2; ++q2) {
        const float4 w = p4[q2];
        const cf w0 = mkcf(w.x, w.y), w1 = mkcf(w.z, w.w);
        a0[2 * q2] = cfmaf(za, w0, a0[2 * q2]);
        a0[2 * q2 + 1] = cfmaf(za, w1, a0[2 * q2 + 1]);
        a1[2 * q2] = cfmaf(zb, w0, a1[2 * q2]);
        a1[2 * q2 + 1] = cfmaf(zb, w1, a1[2 * q2 + 1]);
      }
    } else {
      a0[0] = cfmaf(za, pr[0], a0[0]);
      a1[0] = cfmaf(zb, pr[0], a1[0]);
    }
  }
}

// Same for T rows: only rows >= lo (and < n) are multiplied.
template <int MAXM>
__device__ __forceinline__ void rows_complex_times_from(const cf* __restrict__ Z, int n, int m,
                                                        int ia, int ib, int lo, const cf* P, int ps,
                                                        cf* a0, cf* a1) {
  const bool va = ia < n && ia >= lo, vb = ib < n && ib >= lo;
  for (int qq = 0; qq < m; ++qq) {
    const cf za = va ? Z[ia + (size_t)qq * n] : mkcf(0.f, 0.f);
    const cf zb = vb ? Z[ib + (size_t)qq * n] : mkcf(0.f, 0.f);
    const cf* pr = P + qq * ps;
    if constexpr (MAXM >= 2) {
      const float4* p4 = reinterpret_cast<const float4*>(pr);
#pragma unroll
      for (int q2 = 0; q2 < MAXM / 2; ++q2) {
        const float4 w = p4[q2];
        const cf w0 = mkcf(w.x, w.y), w1 = mkcf(w.z, w.w);
        a0[2 * q2] = cfmaf(za, w0, a0[2 * q2]);
        a0[2 * q2 + 1] = cfmaf(za, w1, a0[2 * q2 + 1]);
        a1[2 * q2] = cfmaf(zb, w0, a1[2 * q2]);
        a1[2 * q2 + 1] = cfmaf(zb, w1, a1[2 * q2 + 1]);
      }
    } else {
      a0[0] = cfmaf(za, pr[0], a0[0]);
      a1[0] = cfmaf(zb, pr[0], a1[0]);
    }
  }
}

// Shifted diagonal of fresh column c (< min(m, nbe)) lies in window row r - m + c.
template <int MAXM>
__device__ __forceinline__ void diag_correction(int ia, int ib, int r, int m, int nbe, cf sigma,
                                                const cf* P, int ps, cf* a0, cf* a1) {
  const int ca = ia - (r - m), cb = ib - (r - m);
  const int lim = min(m, nbe);
  if (ia < r && ca >= 0 && ca < lim) {
    const cf* pr = P + ca * ps;
#pragma unroll
    for (int q = 0; q < MAXM; ++q)
      if (q < m) a0[q] = cfmsf(sigma, pr[q], a0[q]);
  }
  if (ib < r && cb >= 0 && cb < lim) {
    const cf* pr = P + cb * ps;
#pragma unroll
    for (int q = 0; q < MAXM; ++q)
      if (q < m) a1[q] = cfmsf(sigma, pr[q], a1[q]);
  }
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

    // ---- rows above the block, two rows per thread (i, i + kThreads).  With
    // a right-hand side its pass runs first (it reads the old live columns);
    // each thread owns its rows in both passes, so no barrier is needed between.
    if (RHS) {
      for (int i0 = 0; i0 < r; i0 += 2 * kThreads) {
        const int ia = i0 + tid, ib = ia + kThreads;
        cf a0[MAXM], a1[MAXM];
#pragma unroll
        for (int q = 0; q < MAXM; ++q) {
          a0[q] = (ia < r && q < m) ? Zr[ia + (size_t)q * n] : mkcf(0.f, 0.f);
          a1[q] = (ib < r && q < m) ? Zr[ib + (size_t)q * n] : mkcf(0.f, 0.f);
        }
        rows_real_times<MAXM>(Hhi, n, j0, nbe, ia, ib, r, sm.coefr, MAXM, a0, a1);
        rows_complex_times<MAXM>(Zl, n, m, ia, ib, r, sm.coefr + kNB * MAXM, MAXM, a0, a1);
        diag_correction<MAXM>(ia, ib, r, m, nbe, sigma, sm.coefr, MAXM, a0, a1);
#pragma unroll
        for (int q = 0; q < MAXM; ++q) {
          if (q < m) {
            if (ia < r) Zr[ia + (size_t)q * n] = a0[q];
            if (ib < r) Zr[ib + (size_t)q * n] = a1[q];
          }
        }
      }
    }
    for (int i0 = 0; i0 < r; i0 += 2 * kThreads) {
      const int ia = i0 + tid, ib = ia + kThreads;
      cf a0[MAXM], a1[MAXM];
#pragma unroll
      for (int q = 0; q < MAXM; ++q) { a0[q] = mkcf(0.f, 0.f); a1[q] = mkcf(0.f, 0.f); }
      rows_real_times<MAXM>(Hhi, n, j0, nbe, ia, ib, r, sm.coef, S, a0, a1);
      rows_complex_times<MAXM>(Zl, n, m, ia, ib, r, sm.coef + kNB * S, S, a0, a1);
      diag_correction<MAXM>(ia, ib, r, m, nbe, sigma, sm.coef, S, a0, a1);
#pragma unroll
      for (int q = 0; q < MAXM; ++q) {
        if (q < m) {
          if (ia < r) Zl[ia + (size_t)q * n] = a0[q];
          if (ib < r) Zl[ib + (size_t)q * n] = a1[q];
        }
      }
    }
    // ---- T rows j0 .. n-1: fresh rows take the coefficients, the others
    // are multiplied by the old-live block (RHS pass first, as above).
    {
      const int lo = k - m;
      const int nt = n - j0;
      if (RHS) {
        for (int t0 = 0; t0 < nt; t0 += 2 * kThreads) {
          const int ia = j0 + t0 + tid, ib = ia + kThreads;
          cf a0[MAXM], a1[MAXM];
#pragma unroll
          for (int q = 0; q < MAXM; ++q) {
            a0[q] = (ia < n && ia >= lo && q < m) ? Tr[ia + (size_t)q * n] : mkcf(0.f, 0.f);
            a1[q] = (ib < n && ib >= lo && q < m) ? Tr[ib + (size_t)q * n] : mkcf(0.f, 0.f);
          }
          rows_complex_times_from<MAXM>(Tl, n, m, ia, ib, lo, sm.coefr + kNB * MAXM, MAXM, a0, a1);
#pragma unroll
          for (int q = 0; q < MAXM; ++q) {
            if (q < m) {
              if (ia < n) Tr[ia + (size_t)q * n] = ia < lo ? sm.coefr[(ia - j0) * MAXM + q] : a0[q];
              if (ib < n) Tr[ib + (size_t)q * n] = ib < lo ? sm.coefr[(ib - j0) * MAXM + q] : a1[q];
            }
          }
        }
      }
      for (int t0 = 0; t0 < nt; t0 += 2 * kThreads) {
        const int ia = j0 + t0 + tid, ib = ia + kThreads;
        cf a0[MAXM], a1[MAXM];
#pragma unroll
        for (int q = 0; q < MAXM; ++q) { a0[q] = mkcf(0.f, 0.f); a1[q] = mkcf(0.f, 0.f); }
        rows_complex_times_from<MAXM>(Tl, n, m, ia, ib, lo, sm.coef + kNB * S, S, a0, a1);
#pragma unroll
        for (int q = 0; q < MAXM; ++q) {
          if (q < m) {
            if (ia < n) Tl[ia + (size_t)q * n] = ia < lo ? sm.coef[(ia - j0) * S + q] : a0[q];
            if (ib < n) Tl[ib + (size_t)q * n] = ib < lo ? sm.coef[(ib - j0) * S + q] : a1[q];
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

// ---------------------------------------------------------------------------
// Phase kernels.  All per-shift state lives in global arrays indexed by shift
// (Xhat in complex128, E in complex64, flags, eta); the host runs sweep 0,
// then rounds of {residual, check, compact, correction sweep}.  Shifts that are
// finished are dropped from the active list, so later rounds cost one small
// launch each.
// ---------------------------------------------------------------------------
constexpr int kFlagOk = 1;      // converged: backward error <= tol
constexpr int kFlagFail = 2;    // stagnated / iteration limit / singular: FP64 re-solve
constexpr int kFlagSing = 4;    // a finalised diagonal fell below the FP32 threshold
constexpr int kRT = 128;        // residual rows per work item

__device__ __forceinline__ double shifted_norm(const double* hnorm, int n, cd sigma) {
  return sqrt(fmax(hnorm[0] - 2.0 * sigma.x * hnorm[1] +
                       (double)n * (sigma.x * sigma.x + sigma.y * sigma.y), 0.0));
}

// Sweep 0 (RHS = false: Xhat = T(:, live) Wm^{-1} R1) or a correction sweep
// (RHS = true: E, in place, is the dense right-hand side; Xhat += T Y - Tr).
template <int MAXM, bool RHS>
__global__ void __launch_bounds__(kThreads, 2) mixed_sweep_kernel(
    int n, int m, int nb, const float* __restrict__ Hhi, const double* __restrict__ R,
    const cd* __restrict__ shifts, const int* __restrict__ list, const int* __restrict__ count,
    unsigned char* __restrict__ slots, size_t slot_bytes, cd* __restrict__ Xall,
    cf* __restrict__ Eall, int* __restrict__ flags, const double* __restrict__ hnorm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem<MAXM> sm;
  sm.bind(smem_raw);
  __shared__ int s_flag;
  __shared__ int s_piv;
  const int tid = threadIdx.x;
  const size_t nm = (size_t)n * m;
  cf* Zl = reinterpret_cast<cf*>(slots + (size_t)blockIdx.x * slot_bytes);
  cf* Tl = Zl + nm;
  cf* Tr = Tl + nm;
  const int cnt = *count;
  for (int w = blockIdx.x; w < cnt; w += gridDim.x) {
    const int sh = list[w];
    const cd sigma = shifts[sh];
    const cf sigf = mkcf((float)sigma.x, (float)sigma.y);
    const float sing_tol = (float)((double)n * 1.1920928955078125e-07 * shifted_norm(hnorm, n, sigma));
    cf* Zr = Eall + (size_t)sh * nm;
    cd* Xh = Xall + (size_t)sh * nm;
    if (tid == 0) s_flag = 0;
    __syncthreads();
    sweep<MAXM, RHS>(n, m, nb, Hhi, sigf, Zl, Zr, Tl, Tr, sm, sing_tol, &s_flag);
    final_solve<MAXM, RHS>(n, m, Zl, Zr, R, sm, sing_tol, &s_flag, &s_piv);
    for (long long idx = tid; idx < (long long)nm; idx += kThreads) {
      const int i = (int)(idx % n), q = (int)(idx / n);
      float ar = 0.f, ai = 0.f;
      if (RHS) {
        const cf tr = Tr[idx];
        ar = -tr.x;
        ai = -tr.y;
      }
      for (int t = 0; t < m; ++t) {
        const cf a = Tl[i + (size_t)t * n];
        const cf y = sm.yb[t + q * MAXM];
        ar = fmaf(a.x, y.x, fmaf(-a.y, y.y, ar));
        ai = fmaf(a.x, y.y, fmaf(a.y, y.x, ai));
      }
      if (RHS) {
        cd x = Xh[idx];
        x.x += (double)ar;
        x.y += (double)ai;
        Xh[idx] = x;
      } else {
        Xh[idx] = mkcd(ar, ai);
      }
    }
    if (tid == 0 && s_flag) flags[sh] |= kFlagSing;
    __syncthreads();
  }
}

// E = R - (H - sigma I) Xhat for rows [i0, i0 + kRT) of one shift, with
// H = Hhi + Hlo and Xhat split into FP32 pairs, exact FMA products and
// double-float accumulation.  E is stored as complex64; ||E||_F^2 and
// ||Xhat||_F^2 are accumulated per shift in acc (FP64 atomics).
template <int MAXM>
__global__ void __launch_bounds__(kRT, 4) mixed_residual_kernel(
    int n, int m, const float* __restrict__ Hhi, const float* __restrict__ Hlo,
    const double* __restrict__ R, const cd* __restrict__ shifts, const int* __restrict__ list,
    const int* __restrict__ count, const cd* __restrict__ Xall, cf* __restrict__ Eall,
    double* __restrict__ acc) {
  __shared__ float4 xs[kJT * MAXM];
  __shared__ double red[2][kRT / 32];
  const int tid = threadIdx.x;
  const int rt = (n + kRT - 1) / kRT;
  const int cnt = *count;
  const size_t nm = (size_t)n * m;
  for (long long w = blockIdx.x; w < (long long)cnt * rt; w += gridDim.x) {
    const int sh = list[w / rt];
    const int i0 = (int)(w % rt) * kRT;
    const int i = i0 + tid;
    const cd sigma = shifts[sh];
    const cd* Xh = Xall + (size_t)sh * nm;
    float rh[MAXM], rl[MAXM], ih[MAXM], il[MAXM];
#pragma unroll
    for (int q = 0; q < MAXM; ++q) { rh[q] = 0.f; rl[q] = 0.f; ih[q] = 0.f; il[q] = 0.f; }
    const int jlo = max(0, i0 - m);
    for (int jt = jlo; jt < n; jt += kJT) {
      __syncthreads();
      for (int idx = tid; idx < kJT * m; idx += kRT) {
        const int jj = idx % kJT, q = idx / kJT;
        const int j = jt + jj;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n) {
          const cd x = Xh[j + (size_t)q * n];
          const float a = (float)x.x, b = (float)x.y;
          v = make_float4(a, (float)(x.x - (double)a), b, (float)(x.y - (double)b));
        }
        xs[jj * MAXM + q] = v;
      }
      __syncthreads();
      if (i < n) {
        const int jend = min(kJT, n - jt);
        for (int jj0 = 0; jj0 < jend; jj0 += 4) {
          float hh[4], hl[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = jt + jj0 + u;
            hh[u] = 0.f;
            hl[u] = 0.f;
            if (jj0 + u < jend && j >= i - m) {
              hh[u] = Hhi[i + (size_t)j * n];
              hl[u] = Hlo[i + (size_t)j * n];
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
              if (q < m) {
                const float4 x = xs[(jj0 + u) * MAXM + q];
                df_mac(rh[q], rl[q], hh[u], hl[u], x.x, x.y);
                df_mac(ih[q], il[q], hh[u], hl[u], x.z, x.w);
              }
            }
          }
        }
      }
    }
    double e2 = 0.0, x2 = 0.0;
    if (i < n) {
      cf* E = Eall + (size_t)sh * nm;
#pragma unroll
      for (int q = 0; q < MAXM; ++q) {
        if (q < m) {
          const cd x = Xh[i + (size_t)q * n];
          const double hxr = (double)rh[q] + (double)rl[q];
          const double hxi = (double)ih[q] + (double)il[q];
          double er = -hxr + (sigma.x * x.x - sigma.y * x.y);
          double ei = -hxi + (sigma.x * x.y + sigma.y * x.x);
          if (i <= q) er += R[i + (size_t)q * n];
          e2 += er * er + ei * ei;
          x2 += x.x * x.x + x.y * x.y;
          E[i + (size_t)q * n] = mkcf((float)er, (float)ei);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    }
    if ((tid & 31) == 0) {
      red[0][tid >> 5] = e2;
      red[1][tid >> 5] = x2;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < kRT / 32; ++k) { a += red[0][k]; b += red[1][k]; }
      atomicAdd(acc + 2 * (size_t)sh, a);
      atomicAdd(acc + 2 * (size_t)sh + 1, b);
    }
  }
}

// Per active shift: backward error eta from the accumulated norms; decide
// converged (eta <= tol), failed (iteration limit, slow contraction:
// eta > eta_prev / 4, or singular), or another correction.  Resets the
// accumulators.
__global__ void mixed_check_kernel(int n, int m, const double* __restrict__ R,
                                   const cd* __restrict__ shifts, const int* __restrict__ list,
                                   const int* __restrict__ count, double* __restrict__ acc,
                                   double* __restrict__ eta, int* __restrict__ flags,
                                   const double* __restrict__ hnorm, int it, int max_refine,
                                   double tol, const int* __restrict__ err) {
  const int cnt = *count;
  const bool tc_failed = *err != 0;
  double r2 = 0.0;
  for (int q = 0; q < m; ++q)
    for (int i = 0; i <= q; ++i) r2 += R[i + (size_t)q * n] * R[i + (size_t)q * n];
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < cnt; w += gridDim.x * blockDim.x) {
    const int sh = list[w];
    const double mn = shifted_norm(hnorm, n, shifts[sh]);
    const double e2 = acc[2 * (size_t)sh], x2 = acc[2 * (size_t)sh + 1];
    acc[2 * (size_t)sh] = 0.0;
    acc[2 * (size_t)sh + 1] = 0.0;
    const double den = mn * sqrt(x2) + sqrt(r2);
    // NaN (non-finite Xhat) stays NaN and fails below
    const double e = den > 0.0 ? sqrt(e2) / den : (den == den ? 0.0 : den);
    const double prev = eta[sh];
    eta[sh] = e;
    int f = flags[sh];
    // A correction must shrink the backward error by at least 4x (the
    // contraction factor of FP32-based refinement is ~kappa * u32 * growth);
    // slower shifts go to the FP64 sweep at once instead of iterating.
    // a shift flagged singular goes to the FP64 re-solve (which reports it)
    // even when its backward error is small
    if ((f & kFlagSing) || tc_failed) f |= kFlagFail;
    else if (e <= tol) f |= kFlagOk;
    else if (!(e == e) || it >= max_refine || (it > 0 && e > 0.25 * prev)) f |= kFlagFail;
    flags[sh] = f;
  }
}

// Refinement counters on this device (ssv_refine_counts): [0] shift-sweeps of
// correction, [1] shifts handed to the FP64 re-solve.
__device__ unsigned long long g_refine_counts[2];

// Active list: shifts whose flags have neither kFlagOk nor kFlagFail.  With
// `tally`, the shifts listed (those the next correction sweep solves) are
// added to the correction counter.
__global__ void __launch_bounds__(1024) mixed_compact_kernel(int s, const int* __restrict__ flags,
                                                             int* __restrict__ list,
                                                             int* __restrict__ count, int tally) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int chunk = (s + 1023) / 1024;
  const int b = tid * chunk, e = min(s, b + chunk);
  int c = 0;
  for (int j = b; j < e; ++j) c += (flags[j] & (kFlagOk | kFlagFail)) ? 0 : 1;
  part[tid] = c;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {   // inclusive scan
    int v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int pos = part[tid] - c;
  for (int j = b; j < e; ++j)
    if (!(flags[j] & (kFlagOk | kFlagFail))) list[pos++] = j;
  if (tid == 1023) {
    *count = part[1023];
    if (tally) atomicAdd(&g_refine_counts[0], (unsigned long long)part[1023]);
  }
}

// Outputs of converged shifts (G = +-Ct Xhat in FP64, or Xhat); the others are
// marked for the FP64 re-solve.
__global__ void mixed_output_kernel(int n, int m, int p, int s, int mode,
                                    const double* __restrict__ Ct, int ldct,
                                    const cd* __restrict__ Xall, const int* __restrict__ flags,
                                    const double* __restrict__ eta, cd* __restrict__ out,
                                    long long ldo, int* __restrict__ status,
                                    double* __restrict__ resid, int* __restrict__ fallback) {
  const size_t nm = (size_t)n * m;
  for (int sh = blockIdx.x; sh < s; sh += gridDim.x) {
    const bool ok = (flags[sh] & kFlagOk) != 0;
    if (threadIdx.x == 0) {
      fallback[sh] = ok ? 0 : 1;
      if (!ok) atomicAdd(&g_refine_counts[1], 1ull);
      if (ok && status) status[sh] = SSV_SHIFT_OK;
      if (ok && resid) resid[sh] = eta[sh];
    }
    if (!ok) continue;
    const cd* Xh = Xall + (size_t)sh * nm;
    cd* o = out + (size_t)sh * m * ldo;
    if (mode == SSV_G || mode == SSV_TF) {
      const double sg = mode == SSV_TF ? -1.0 : 1.0;
      for (int idx = threadIdx.x; idx < p * m; idx += blockDim.x) {
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
      for (long long idx = threadIdx.x; idx < (long long)nm; idx += blockDim.x) {
        const int i = (int)(idx % n), q = (int)(idx / n);
        o[i + (size_t)q * ldo] = Xh[idx];
      }
    }
  }
}

__global__ void mixed_init_kernel(int s, int* __restrict__ flags, double* __restrict__ eta,
                                  double* __restrict__ acc, int* __restrict__ list,
                                  int* __restrict__ count) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x) {
    flags[j] = 0;
    eta[j] = INFINITY;
    acc[2 * (size_t)j] = 0.0;
    acc[2 * (size_t)j + 1] = 0.0;
    list[j] = j;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = s;
}

// Statuses of the first solve -> flags (singular or non-finite shifts go to
// the FP64 re-solve like every other failure).
__global__ void mixed_status_kernel(int s, const int* __restrict__ st0, int* __restrict__ flags) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < s; j += gridDim.x * blockDim.x)
    if (st0[j] != SSV_SHIFT_OK) flags[j] |= kFlagSing;
}

// Scratch of one mixed solve, carved from one stream-ordered allocation.
struct MixedScratch {
  cd* X;         // s * n * m
  cf* E;         // s * n * m
  unsigned char* slots;  // grid * slot_bytes
  double* acc;   // 2 s
  double* eta;   // s
  int* flags;    // s
  int* list;     // s
  int* fallback; // s
  int* st0;      // s: statuses of the first (double-float) solve
  int* count;    // 1
  int* err;      // 1: a tensor-core residual wait gave up
  unsigned char* tch;  // digit slices of H (tensor-core residual, m <= 16), or null
  unsigned char* tcx;  // digit slices of Xhat for s shifts, or null
  size_t bytes;
};

size_t mixed_layout(int n, int m, int s, int grid, size_t slot_bytes, MixedScratch* ms,
                    unsigned char* base) {
  size_t off = 0;
  auto take = [&](size_t b) {
    size_t o = off;
    off += (b + 255) / 256 * 256;
    return o;
  };
  const size_t nm = (size_t)n * m;
  size_t oX = take(sizeof(cd) * nm * s), oE = take(sizeof(cf) * nm * s);
  size_t oS = take(slot_bytes * grid), oA = take(sizeof(double) * 2 * s),
         oT = take(sizeof(double) * s), oF = take(sizeof(int) * s), oL = take(sizeof(int) * s),
         oB = take(sizeof(int) * s), oS0 = take(sizeof(int) * s), oC = take(sizeof(int)),
         oR = take(sizeof(int));
  const bool tc = m <= kTcMaxM;
  const size_t oH = tc ? take(resid_tc_hbytes(n)) : 0, oXs = tc ? take(resid_tc_xbytes(n, s)) : 0;
  if (ms && base) {
    ms->X = reinterpret_cast<cd*>(base + oX);
    ms->E = reinterpret_cast<cf*>(base + oE);
    ms->slots = base + oS;
    ms->acc = reinterpret_cast<double*>(base + oA);
    ms->eta = reinterpret_cast<double*>(base + oT);
    ms->flags = reinterpret_cast<int*>(base + oF);
    ms->list = reinterpret_cast<int*>(base + oL);
    ms->fallback = reinterpret_cast<int*>(base + oB);
    ms->st0 = reinterpret_cast<int*>(base + oS0);
    ms->count = reinterpret_cast<int*>(base + oC);
    ms->err = reinterpret_cast<int*>(base + oR);
    ms->tch = tc ? base + oH : nullptr;
    ms->tcx = tc ? base + oXs : nullptr;
    ms->bytes = off;
  }
  return off;
}

constexpr int kSweepBlocksPerSm = 2;
constexpr int kResidBlocksPerSm = 8;

template <int MAXM>
int run_mixed(const Handle* h, int s, const double* shifts, int nb, int mode, double* out,
              long long ldo, int* status, double* resid, int max_refine, double tol, int first,
              int** fallback_out, void** scratch_out, cudaStream_t st) {
  using L = LayoutM<MAXM>;
  const int n = h->n, m = h->m, p = h->p;
  const size_t slot_bytes = (size_t)n * m * 3 * sizeof(cf);
  auto k1 = mixed_sweep_kernel<MAXM, true>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
  int occ1 = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k1, kThreads, L::bytes));
  const int per_sm = std::max(1, std::min(occ1, kSweepBlocksPerSm));
  const int grid = std::max(1, std::min(s, num_sms() * per_sm));
  const size_t total = mixed_layout(n, m, s, grid, slot_bytes, nullptr, nullptr);
  unsigned char* base = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&base, total, st));
  *scratch_out = base;
  MixedScratch ms;
  mixed_layout(n, m, s, grid, slot_bytes, &ms, base);
  *fallback_out = ms.fallback;
  const cd* sd = reinterpret_cast<const cd*>(shifts);
  mixed_init_kernel<<<std::min(1024, (s + 255) / 256), 256, 0, st>>>(s, ms.flags, ms.eta, ms.acc,
                                                                     ms.list, ms.count);
  count_launch();
  // first solve: the double-float sweep (double-word panels, FP32-pair bulk
  // updates) writes Xhat of every shift and flags its singular shifts.  With
  // SSV_FIRST_C64 Xhat starts at zero instead: the residual of the round
  // numbered -1 below is then R itself, and that round's correction sweep is
  // the complex64 first solve.
  const bool c64 = first == SSV_FIRST_C64;
  const bool tens = first == SSV_FIRST_TENSOR && ms.tch != nullptr && solve_tc_supported(h, SSV_XHAT);
  bool h_split = false;
  if (tens) {
    // the H digit tiles serve the tensor-core sweep and then the residual
    void* trs = trace_begin("mixed_split_h", st);
    const int rc = resid_tc_split_h(h, ms.tch, st);
    trace_end(trs, st);
    if (rc != SSV_OK) return rc;
    h_split = true;
  }
  void* tr = trace_begin("mixed_sweep0", st);
  if (c64) {
    SSV_CUDA_TRY(cudaMemsetAsync(ms.X, 0, sizeof(cd) * (size_t)n * m * s, st));
  } else if (tens) {
    const int rc0 = solve_tc(h, s, shifts, SSV_XHAT, reinterpret_cast<double*>(ms.X), n, ms.st0,
                             ms.tch, st);
    if (rc0 != SSV_OK) return rc0;
    mixed_status_kernel<<<std::min(1024, (s + 255) / 256), 256, 0, st>>>(s, ms.st0, ms.flags);
    count_launch();
  } else {
    ssv_opts od;
    ssv_default_opts(&od);
    od.precision = SSV_DFLOAT;
    od.mode = SSV_XHAT;
    int rc0 = solve_fp64(h, s, shifts, &od, reinterpret_cast<double*>(ms.X), n, ms.st0, nullptr, st);
    if (rc0 != SSV_OK) return rc0;
    mixed_status_kernel<<<std::min(1024, (s + 255) / 256), 256, 0, st>>>(s, ms.st0, ms.flags);
    count_launch();
  }
  trace_end(tr, st);
  const int rgrid = num_sms() * kResidBlocksPerSm;
  SSV_CUDA_TRY(cudaMemsetAsync(ms.err, 0, sizeof(int), st));
  if (ms.tch != nullptr && !h_split) {
    tr = trace_begin("mixed_split_h", st);
    const int rc = resid_tc_split_h(h, ms.tch, st);
    trace_end(tr, st);
    if (rc != SSV_OK) return rc;
  }
  for (int it = c64 ? -1 : 0; it <= max_refine; ++it) {
    tr = trace_begin("mixed_residual", st);
    if (ms.tch != nullptr) {
      // Ozaki-split BF16 products on the tensor cores (residual_tc.cu)
      const int rc = resid_tc_run(h, ms.tch, ms.tcx, s, shifts, ms.list, ms.count,
                                  reinterpret_cast<const double*>(ms.X), n, ms.E, ms.acc, ms.err, st);
      if (rc != SSV_OK) return rc;
    } else {
      mixed_residual_kernel<MAXM><<<rgrid, kRT, 0, st>>>(n, m, h->Hhi, h->Hlo, h->R, sd, ms.list,
                                                        ms.count, ms.X, ms.E, ms.acc);
      count_launch();
    }
    trace_end(tr, st);
    mixed_check_kernel<<<std::min(1024, (s + 255) / 256), 256, 0, st>>>(
        n, m, h->R, sd, ms.list, ms.count, ms.acc, ms.eta, ms.flags, h->hnorm2, it, max_refine, tol,
        ms.err);
    count_launch();
    mixed_compact_kernel<<<1, 1024, 0, st>>>(s, ms.flags, ms.list, ms.count,
                                             (it >= 0 && it < max_refine) ? 1 : 0);
    count_launch();
    if (it == max_refine) break;
    tr = trace_begin(it < 0 ? "mixed_first_c64" : "mixed_correction", st);
    k1<<<grid, kThreads, L::bytes, st>>>(n, m, nb, h->Hhi, h->R, sd, ms.list, ms.count, ms.slots,
                                        slot_bytes, ms.X, ms.E, ms.flags, h->hnorm2);
    count_launch();
    trace_end(tr, st);
  }
  mixed_output_kernel<<<std::min(s, num_sms() * 8), 256, 0, st>>>(
      n, m, p, s, mode, h->Ct, p > 0 ? p : 1, ms.X, ms.flags, ms.eta,
      reinterpret_cast<cd*>(out), ldo, status, resid, ms.fallback);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

}  // namespace

int refine_counts(long long c[2], bool reset) {
  unsigned long long v[2] = {0, 0};
  SSV_CUDA_TRY(cudaMemcpyFromSymbol(v, g_refine_counts, sizeof(v)));
  if (reset) {
    const unsigned long long z[2] = {0, 0};
    SSV_CUDA_TRY(cudaMemcpyToSymbol(g_refine_counts, z, sizeof(z)));
  }
  c[0] = (long long)v[0];
  c[1] = (long long)v[1];
  return SSV_OK;
}

size_t solve_mixed_scratch_bytes(int n, int m, int p, int s, const ssv_opts* o) {
  const size_t slot_bytes = (size_t)n * m * 3 * sizeof(cf);
  const int grid = std::max(1, std::min(s, num_sms() * kSweepBlocksPerSm));
  size_t b = mixed_layout(n, m, s, grid, slot_bytes, nullptr, nullptr) + 256;
  // the tensor-core first solve allocates its own window state while it runs
  if (o->first == SSV_FIRST_TENSOR && m <= kTcMaxM && n > m)
    b += solve_tc_scratch_bytes(n, m, p, s, SSV_XHAT);
  return b;
}

int solve_mixed(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                long long ldo, int* status, double* resid, cudaStream_t st) {
  const int m = h->m;
  const int nb = o->nb > 0 ? o->nb : std::min(kNB, tuned_nb(h->n, m, h->p, SSV_MIXED, o->mode));
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  int* fallback = nullptr;
  void* scratch = nullptr;
  int rc;
  const int mode = o->mode == SSV_X ? SSV_XHAT : o->mode;
  const int mr = o->max_refine;
  const double tol = o->tol;
  if (m <= 1) rc = run_mixed<1>(h, s, shifts, nb, mode, out, ldo, status, resid, mr, tol, o->first, &fallback, &scratch, st);
  else if (m <= 2) rc = run_mixed<2>(h, s, shifts, nb, mode, out, ldo, status, resid, mr, tol, o->first, &fallback, &scratch, st);
  else if (m <= 4) rc = run_mixed<4>(h, s, shifts, nb, mode, out, ldo, status, resid, mr, tol, o->first, &fallback, &scratch, st);
  else if (m <= 8) rc = run_mixed<8>(h, s, shifts, nb, mode, out, ldo, status, resid, mr, tol, o->first, &fallback, &scratch, st);
  else if (m <= 16) rc = run_mixed<16>(h, s, shifts, nb, mode, out, ldo, status, resid, mr, tol, o->first, &fallback, &scratch, st);
  else if (m <= 32) rc = run_mixed<32>(h, s, shifts, nb, mode, out, ldo, status, resid, mr, tol, o->first, &fallback, &scratch, st);
  else rc = SSV_ENOTSUP;
  // shifts that did not converge: FP64 sweep (status and output overwritten);
  // their backward errors come from the FP64 solution
  if (rc == SSV_OK && resid == nullptr) {
    void* tr = trace_begin("mixed_fallback", st);
    rc = solve_fp64_masked(h, s, shifts, mode, 0, out, ldo, status, fallback, nullptr, 0, st);
    trace_end(tr, st);
  }
  if (rc == SSV_OK && resid != nullptr) {
    cd* xcopy = nullptr;
    const bool gm = (mode == SSV_G || mode == SSV_TF);
    if (gm) {
      cudaError_t e = pool_alloc((void**)&xcopy, sizeof(cd) * (size_t)h->n * m * s, st);
      if (e != cudaSuccess) { set_cuda_error(e); rc = SSV_ENOMEM; }
    }
    if (rc == SSV_OK)
      rc = solve_fp64_masked(h, s, shifts, mode, 0, out, ldo, status, fallback, xcopy, h->n, st);
    if (rc == SSV_OK)
      rc = backward_error_fp64_masked(h, s, shifts, gm ? reinterpret_cast<const double*>(xcopy) : out,
                                      gm ? h->n : ldo, resid, fallback, st);
    if (xcopy) cudaFreeAsync(xcopy, st);
  }
  if (scratch) {
    cudaError_t e = cudaFreeAsync(scratch, st);
    if (e != cudaSuccess && rc == SSV_OK) {
      set_cuda_error(e);
      rc = SSV_ECUDA;
    }
  }
  return rc;
}

}  // namespace ssv
