// Persistent shift-batched solver for (H - sigma I) Xhat = R, FP64.
//
// The method is the blocked bottom-up elimination of Sec. 3.1 / Algorithm 8:
// a sliding window of the columns of [Ct; H - sigma I] moves from the last
// column to the first.  Its "live" part Z2 (m columns, specific to the shift)
// is combined with n_b fresh columns Z1 of the original [Ct; H] (shared by all
// shifts) on each block of n_b rows:
//   1. the n_b x (n_b + m) window block is triangularised from its bottom row
//      up.  Row c has m + 1 candidate entries (m live columns and the fresh
//      column that enters at this row); one complex Householder reflector
//      acting on those m + 1 columns from the right maps the row onto the
//      fresh column's slot (an RQ step, as in Sec. 3.1).  The reflector is
//      applied to the rows of the block above c and accumulated into the
//      coefficients P ((n_b + m) x m) that express the m surviving columns in
//      terms of [Z1 | Z2]; the rest of the block transform is never formed,
//      the economy of Sec. 3.1;
//   2. the rows above the block are updated once:
//      Z2 <- Z1 P(1:n_b, :) + Z2 P(n_b+1:, :) - sigma E P(1:min(m,n_b), :),
//      the last term being the shifted diagonal of the fresh columns that
//      lies above the block (Algorithm 8, diagonal correction);
//   3. the window slides up by n_b rows.
// When m rows remain, the live block W = [Wc; Wm] (p + m rows) gives
// Y = Wm^{-1} R(1:m, 1:m) (Gauss-Jordan with partial pivoting) and G = Wc Y
// (Algorithm 8, final loop; here on the GPU).  For Xhat the window also
// carries the rows of the accumulated column transformation T (the "Q*" rows
// of Sec. 3.3), Xhat = T(:, live) Y.  With one right-hand side R bhat_l per
// shift (Sec. 3.3) Y is the m-vector Wm^{-1} R(1:m, 1:m) bhat_l.
//
// Differences from the paper: one Householder reflector per row instead of
// the Givens schedule (unitary either way, so the one-shot update of the rows
// above stays stable); each thread block owns one shift at a time for the
// whole sweep (no grid-wide phases); the final m x m solve runs on the GPU.
#include <algorithm>
#include <map>
#include <tuple>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "dfloat.cuh"
#include "ssv_internal.cuh"

namespace ssv {

namespace {

constexpr int kThreads = 256;
constexpr int kNB = 128;  // maximum rows per block (runtime nb <= kNB)

// Shared memory per thread block:
//   cand[slot * kNB + t]       rows t of the window block, slot in [0, m]
//   coef[c * (MAXM + 1) + slot] coefficient of window column c (fresh c < kNB,
//                               old live kNB + q) in candidate column `slot`
//   Wm, lmul, Yb               final m x m solve
template <int MAXM>
struct Layout {
  static constexpr int kSlots = MAXM + 2;
  static constexpr int kCoefRows = kNB + MAXM;
  static constexpr size_t cand_elems = (size_t)kSlots * kNB;
  static constexpr size_t coef_elems = (size_t)kCoefRows * kSlots;
  // + the dense right-hand side's block rows and coefficients (RHS sweeps)
  static constexpr size_t bytes =
      (cand_elems + coef_elems + 3 * MAXM * MAXM + 2 * MAXM + 4 + kNB + kCoefRows) * sizeof(cd) + 64;
};

// Givens-panel variant (Sec. 3.2, Algorithms 9/10): the whole window block
// Zb (n_b x (n_b + m), column-major, ld kNBG) and its column transform P
// ((n_b + m) x (n_b + m), ld kNBG + MAXM) live in shared memory, so
// n_b <= kNBG; coefficient rows: fresh c < kNBG, old live kNBG + q.
constexpr int kNBG = 32;
template <int MAXM>
struct GivensLayout {
  static constexpr int kSlots = MAXM + 2;
  static constexpr int kCols = kNBG + MAXM;
  static constexpr int kCoefRows = kNBG + MAXM;
  static constexpr size_t zb_elems = (size_t)kNBG * kCols;
  static constexpr size_t p_elems = (size_t)kCols * kCols;
  static constexpr size_t coef_elems = (size_t)kCoefRows * kSlots;
  static constexpr size_t bytes =
      (zb_elems + p_elems + coef_elems + 3 * MAXM * MAXM + 2 * MAXM + 4 + 2 * kNBG) * sizeof(cd) +
      kNBG * sizeof(int) + 64;
};

// Greedy annihilation schedule of one block shape (n_b rows, n_b + m columns):
// rotation j zeroes (r, c1) of the block with (r, c2), packed r | c1 << 8 |
// c2 << 16 (0-based); step t holds rotations off[t] .. off[t+1]-1.
struct GivensSched {
  const int* rot;
  const int* off;
  int nsteps;
};

// One system as the FP64 solve sees it.
struct FpSys {
  int n, m, p, nb, mode;
  const double* H;
  const double* Ct;
  int ldct;
  const double* R;
  const cd* shifts;
  cd* out;
  long long ldo;
  int* status;
  cd* xhat_copy;
  long long ldxc;
  const double* hnorm;
  const cd* bhat;    // per-shift right-hand side coefficients (m x s, ld ldb), or null
  long long ldb;
  const cd* rhs;     // dense right-hand sides (n x s, ld ldr) of an RHS sweep (p == 0)
  long long ldr;
  int flip_out;      // write output row i to row n-1-i (transposed systems)
  const float* Hhi;   // double-float split of H (SSV_DFLOAT updates)
  const float* Hlo;
  GivensSched gfull;  // Givens panel: schedule of full blocks (n_b rows)
  GivensSched gtail;  // and of the last, shorter block
};

// Solve shift sh of system d with the window state in Z2 (and ZT).  With RHS,
// the dense right-hand side d.rhs(:, sh) is carried through the sweep: each
// finalised column F_c (diagonal beta_c) removes f_c = rhs_c / beta_c times
// itself from the rows above (back substitution against the triangular factor
// as it is produced, bottom-up), the rows above the block through the
// accumulated coefficients `coefr`; the solution is T(:, live) y - Tr with Tr
// the T rows of sum_c (-f_c) F_c and y from the final m x m block.
template <int MAXM, bool RHS = false, bool GIVENS = false, bool DF = false>
__device__ void fp64_shift(const FpSys& d, const int sh, cd* __restrict__ Z2,
                           unsigned char* smem_raw, int* s_piv_p, int* s_sing_p) {
  using L = Layout<MAXM>;
  using GL = GivensLayout<MAXM>;
  constexpr int S = L::kSlots;
  constexpr int LB = GIVENS ? kNBG : kNB;   // coefficient row of old live column 0
  constexpr int CR = GIVENS ? GL::kCoefRows : L::kCoefRows;
  cd* cand = reinterpret_cast<cd*>(smem_raw);
  cd* Zb = cand;                             // Givens: window block
  cd* Pg = Zb + GL::zb_elems;                // Givens: column transform
  cd* coef = GIVENS ? Pg + GL::p_elems : cand + L::cand_elems;
  cd* Wm = coef + (GIVENS ? GL::coef_elems : L::coef_elems);  // MAXM x (2 MAXM) augmented [Wm | R1]
  cd* lmul = Wm + 2 * MAXM * MAXM;           // reflector v (MAXM + 2 slots) and tau
  cd* Yb = lmul + (MAXM + 4);                // MAXM x MAXM solution
  cd* rhs_s = Yb + MAXM * MAXM;              // RHS rows of the block (kNB)
  cd* coefr = rhs_s + kNB;                   // RHS coefficients (kCoefRows)
  cd* grot = Yb + MAXM * MAXM;               // Givens: (g0, g1) of the step's rotations
  int* grc = reinterpret_cast<int*>(grot + 2 * kNBG);  // Givens: packed (r, c1, c2)
  int& s_piv = *s_piv_p;
  int& s_sing = *s_sing_p;
  const int n = d.n, m = d.m, p = d.p, nb = d.nb, mode = d.mode, ldct = d.ldct;
  const double* __restrict__ H = d.H;
  const double* __restrict__ Ct = d.Ct;
  const double* __restrict__ R = d.R;
  const cd* __restrict__ shifts = d.shifts;
  cd* __restrict__ out = d.out;
  const long long ldo = d.ldo, ldxc = d.ldxc;
  int* __restrict__ status = d.status;
  cd* __restrict__ xhat_copy = d.xhat_copy;
  const double* __restrict__ hnorm = d.hnorm;
  const int tid = threadIdx.x;
  const int ldz = p + n;
  const bool track_t = RHS || (mode == SSV_XHAT || mode == SSV_X || xhat_copy != nullptr);
  cd* ZT = Z2 + (size_t)ldz * m;  // n x m, valid when track_t
  cd* Zr = ZT + (size_t)n * m;    // RHS rows in progress (n), when RHS
  cd* Tr = Zr + n;                // T rows of the removed finalised columns (n), when RHS
  // With double-float updates the window state Z2 is kept as FP32 pairs
  // (one float4 per complex entry, the size of a complex128), so the bulk
  // update reads and writes it without FP64 conversions.
  float4* const Z2f = reinterpret_cast<float4*>(Z2);
  auto z2ld = [&](size_t idx) -> cd {
    if constexpr (DF) return df_join(Z2f[idx]);
    else return Z2[idx];
  };
  auto z2st = [&](size_t idx, cd v) {
    if constexpr (DF) Z2f[idx] = df_split(v);
    else Z2[idx] = v;
  };
  const cd sigma = shifts[sh];
  // ||H - sigma I||_F from ||H||_F^2 and trace(H); a finalized diagonal entry
  // of magnitude <= n eps ||H - sigma I||_F marks the shift singular.
  const double mnorm2 = fmax(hnorm[0] - 2.0 * sigma.x * hnorm[1] +
                                 (double)n * (sigma.x * sigma.x + sigma.y * sigma.y), 0.0);
  // (with double-float bulk updates the working precision is 2^-47)
  const double sing_tol = (double)n * (DF ? 7.105427357601002e-15 : 2.220446049250313e-16) * sqrt(mnorm2);
  // ---- shift setup: Z2 = last m columns of [Ct; H] - sigma on the diagonal
  for (long long idx = tid; idx < (long long)ldz * m; idx += kThreads) {
    int i = (int)(idx % ldz), q = (int)(idx / ldz);
    int j = n - m + q;
    double v = i < p ? Ct[i + (size_t)j * ldct] : H[(i - p) + (size_t)j * n];
    cd z = mkcd(v, 0.0);
    if (i - p == j) z = csub(z, sigma);
    z2st(idx, z);
  }
  if (track_t) {
    for (long long idx = tid; idx < (long long)n * m; idx += kThreads) {
      int i = (int)(idx % n), q = (int)(idx / n);
      ZT[idx] = mkcd(i == n - m + q ? 1.0 : 0.0, 0.0);
    }
  }
  if (RHS) {
    const cd* rin = d.rhs + (size_t)sh * d.ldr;
    for (int i = tid; i < n; i += kThreads) {
      Zr[i] = rin[i];
      Tr[i] = mkcd(0.0, 0.0);
    }
  }
  if (tid == 0) s_sing = 0;
  __syncthreads();

  // Deferred T rows (X-hat output without per-step T updates).  The rows of
  // the accumulated column transform T set at block step b are P1_b, and
  // every later step multiplies all rows set before it by its P2, so
  //   X-hat(rows of step b) = P1_b P2_{b+1} ... P2_B Y,
  // which a backward pass z_B = Y, X-hat_b = P1_b z_b, z_{b-1} = P2_b z_b
  // forms in O(n m^2) instead of O(n^2 m^2 / n_b) updates.  P1_b stays in ZT;
  // P2_b (m x m) is parked in this shift's own output rows n - b m ..
  // n - (b - 1) m - 1, which the backward pass reaches only after reading it
  // when n_b >= m.
  const bool defer_t = track_t && !RHS && d.bhat == nullptr && !d.flip_out && nb >= m;
  cd* const tout = (mode == SSV_XHAT || mode == SSV_X) ? out + (size_t)sh * m * ldo
                                                        : (xhat_copy != nullptr ? xhat_copy + (size_t)sh * m * ldxc : nullptr);
  const long long tld = (mode == SSV_XHAT || mode == SSV_X) ? ldo : ldxc;
  int nsteps = 0;

  int k = n;
  while (k > m) {
    ++nsteps;
    const int nbe = min(nb, k - m);
    const int r = p + k - nbe;        // rows of [Ct; M] above the block
    const int j0 = k - m - nbe;       // first fresh column
    if constexpr (GIVENS) {
      // ---- RQ of the window block with the greedy Givens schedule
      const int nc = nbe + m;
      constexpr int ldp = GL::kCols;
      for (int idx = tid; idx < nc * nbe; idx += kThreads) {
        const int t = idx % nbe, col = idx / nbe;
        cd z;
        if (col < nbe) {  // fresh column j0 + col: nonzero in block rows t <= col
          z = mkcd(t <= col ? H[(k - nbe + t) + (size_t)(j0 + col) * n] : 0.0, 0.0);
          if (t == col - m) z = csub(z, sigma);
        } else {
          z = Z2[(r + t) + (size_t)(col - nbe) * ldz];
        }
        Zb[col * kNBG + t] = z;
      }
      for (int idx = tid; idx < nc * nc; idx += kThreads) {
        const int row = idx % nc, col = idx / nc;
        Pg[col * ldp + row] = mkcd(row == col ? 1.0 : 0.0, 0.0);
      }
      __syncthreads();
      const GivensSched& gs = (nbe == nb) ? d.gfull : d.gtail;
      for (int step = 0; step < gs.nsteps; ++step) {
        const int j0r = gs.off[step], cnt = gs.off[step + 1] - j0r;
        // rotation j maps [a, b] = Zb(r, (c1, c2)) to [0, rho]:
        // G = [[g0, conj(g1)], [-g1, conj(g0)]], g0 = b / rho, g1 = a / rho
        for (int j = tid; j < cnt; j += kThreads) {
          const int pk = gs.rot[j0r + j];
          const int rr = pk & 255, c1 = (pk >> 8) & 255, c2 = (pk >> 16) & 255;
          const cd a = Zb[c1 * kNBG + rr], b = Zb[c2 * kNBG + rr];
          const double rho = hypot(hypot(a.x, a.y), hypot(b.x, b.y));
          cd g0 = mkcd(1.0, 0.0), g1 = mkcd(0.0, 0.0);
          if (rho > 0.0) {
            g0 = mkcd(b.x / rho, b.y / rho);
            g1 = mkcd(a.x / rho, a.y / rho);
          }
          grot[2 * j] = g0;
          grot[2 * j + 1] = g1;
          grc[j] = pk;
        }
        __syncthreads();
        // [x1, x2] <- [x1 g0 - x2 g1, x1 conj(g1) + x2 conj(g0)] on the block rows
        // 0 .. r and on every row of P
        const int span = nbe + nc;
        for (int e = tid; e < cnt * span; e += kThreads) {
          const int j = e / span, w = e % span;
          const int pk = grc[j];
          const int rr = pk & 255, c1 = (pk >> 8) & 255, c2 = (pk >> 16) & 255;
          cd *x1, *x2;
          if (w < nbe) {
            if (w > rr) continue;
            x1 = Zb + c1 * kNBG + w;
            x2 = Zb + c2 * kNBG + w;
          } else {
            x1 = Pg + c1 * ldp + (w - nbe);
            x2 = Pg + c2 * ldp + (w - nbe);
          }
          const cd g0 = grot[2 * j], g1 = grot[2 * j + 1];
          const cd u = *x1, v = *x2;
          const cd nu = csub(cmul(u, g0), cmul(v, g1));
          const cd nv = cfma(u, mkcd(g1.x, -g1.y), cmul(v, mkcd(g0.x, -g0.y)));
          *x1 = (w == rr) ? mkcd(0.0, 0.0) : nu;
          *x2 = nv;
        }
        __syncthreads();
      }
      // R(t, t + m) is the finalised diagonal of block row t
      for (int t = tid; t < nbe; t += kThreads) {
        const cd dgl = Zb[(t + m) * kNBG + t];
        if (sqrt(dgl.x * dgl.x + dgl.y * dgl.y) <= sing_tol) s_sing = 1;
      }
      // the first m columns of P express the surviving (new live) columns:
      // coefficient rows fresh c -> P(c, q), old live qq -> P(nbe + qq, q)
      for (int idx = tid; idx < CR * S; idx += kThreads) {
        const int crow = idx / S, q = idx % S;
        cd v = mkcd(0.0, 0.0);
        if (q < m) {
          if (crow < nbe) v = Pg[q * ldp + crow];
          else if (crow >= LB && crow - LB < m) v = Pg[q * ldp + nbe + (crow - LB)];
        }
        coef[idx] = v;
      }
      __syncthreads();
    } else if constexpr (DF) {
      // ---- panel in double-float: the window block `cand` and the
      // coefficients `coef` are held as FP32 pairs (re_hi, re_lo, im_hi, im_lo);
      // each row's reflector is formed from them in double-word scalars and
      // applied in double-float, all on the FP32 pipe.
      float4* cand4 = reinterpret_cast<float4*>(cand);
      float4* coef4 = reinterpret_cast<float4*>(coef);
      float4* vf = reinterpret_cast<float4*>(Yb);  // reflector v and tau (slot MAXM + 2)
      const float sing_tol_f = (float)sing_tol;
      static_assert(kNB <= kThreads, "one thread per prefetched fresh entry");
      auto split4 = [](cd z) -> float4 {
        const float rh = (float)z.x, ih = (float)z.y;
        return make_float4(rh, (float)(z.x - (double)rh), ih, (float)(z.y - (double)ih));
      };
      // entry (global row gr, fresh column jc) of H - sigma I as FP32 pairs
      auto fresh4 = [&](int gr, int jc) -> float4 {
        const size_t hidx = (size_t)gr + (size_t)jc * n;
        if (gr == jc) return split4(csub(mkcd((double)d.Hhi[hidx] + (double)d.Hlo[hidx], 0.0), sigma));
        return make_float4(d.Hhi[hidx], d.Hlo[hidx], 0.f, 0.f);
      };
      for (int idx = tid; idx < m * nbe; idx += kThreads) {
        int t = idx % nbe, q = idx / nbe;
        cand4[q * kNB + t] = Z2f[(r + t) + (size_t)q * ldz];
      }
      for (int idx = tid; idx < L::kCoefRows * S; idx += kThreads) {
        int c = idx / S, slot = idx % S;
        const bool one = (slot < m && c == kNB + slot) || (slot == m && c == nbe - 1);
        coef4[idx] = make_float4(one ? 1.f : 0.f, 0.f, 0.f, 0.f);
      }
      {
        const int c = nbe - 1, jc = j0 + c;
        for (int t = tid; t <= c; t += kThreads) cand4[m * kNB + t] = fresh4(k - nbe + t, jc);
      }
      __syncthreads();
      for (int c = nbe - 1; c >= 0; --c) {
        const int fs = m + ((nbe - 1 - c) & 1);
        const int fn = (fs == m) ? m + 1 : m;
        // the next fresh column is read from H now, its latency hidden behind
        // this row's reflector and update (H is not written by the sweep)
        float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c > 0 && tid < c) pre = fresh4(k - nbe + tid, j0 + c - 1);
        if (tid < 32) {
          // reflector scalars in double-word arithmetic:
          //   v = conj(x) + e^{i arg conj(x_f)} ||x|| e_f,  tau = 1 / (||x||^2 + |x_f| ||x||)
          dw rest2{0.f, 0.f};
          for (int q = tid; q < m; q += 32) {
            const float4 x = cand4[q * kNB + c];
            df_mac(rest2.hi, rest2.lo, x.x, x.y, x.x, x.y);
            df_mac(rest2.hi, rest2.lo, x.z, x.w, x.z, x.w);
            vf[q] = make_float4(x.x, x.y, -x.z, -x.w);
          }
          rest2 = dw_fast(rest2.hi, rest2.lo);
          for (int o = 16; o > 0; o >>= 1)
            rest2 = dw_add(rest2, dw{__shfl_xor_sync(0xffffffffu, rest2.hi, o),
                                     __shfl_xor_sync(0xffffffffu, rest2.lo, o)});
          if (tid == 0) {
            const float4 xf = cand4[fs * kNB + c];
            const dw xr{xf.x, xf.y}, xi{xf.z, xf.w};
            const dw af2 = dw_add(dw_mul(xr, xr), dw_mul(xi, xi));
            const dw af = dw_sqrt(af2);
            const dw nrm2 = dw_add(rest2, af2);
            const dw nrm = dw_sqrt(nrm2);
            float4 vfs;
            if (af.hi > 0.f) {  // conj(x_f) (1 + ||x|| / |x_f|)
              const dw g = dw_add(dw{1.f, 0.f}, dw_div(nrm, af));
              const dw vr = dw_mul(xr, g), vi = dw_mul(xi, g);
              vfs = make_float4(vr.hi, vr.lo, -vi.hi, -vi.lo);
            } else {
              vfs = make_float4(nrm.hi, nrm.lo, 0.f, 0.f);
            }
            vf[fs] = vfs;
            const dw tau = rest2.hi > 0.f ? dw_div(dw{1.f, 0.f}, dw_add(nrm2, dw_mul(af, nrm)))
                                          : dw{0.f, 0.f};
            vf[MAXM + 2] = make_float4(tau.hi, tau.lo, 0.f, 0.f);
            if (nrm.hi <= sing_tol_f) s_sing = 1;
          }
        }
        __syncthreads();
        const float4 tauf = vf[MAXM + 2];
        if (tauf.x != 0.0f) {
          const int nrow = c;
          const int ncoef = (nbe - c) + m;
          for (int e = tid; e < nrow + ncoef; e += kThreads) {
            float4* base;
            int stride;
            if (e < nrow) {
              base = cand4 + e;
              stride = kNB;
            } else {
              const int ee = e - nrow;
              const int crow = ee < nbe - c ? c + ee : kNB + (ee - (nbe - c));
              base = coef4 + crow * S;
              stride = 1;
            }
            // w = sum_slot base(slot) v(slot)
            float wrh = 0.f, wrl = 0.f, wih = 0.f, wil = 0.f;
            for (int q = 0; q <= m; ++q) {
              const int slot = q < m ? q : fs;
              const float4 x = base[slot * stride], v = vf[slot];
              df_mac(wrh, wrl, x.x, x.y, v.x, v.y);
              df_mac(wrh, wrl, -x.z, -x.w, v.z, v.w);
              df_mac(wih, wil, x.x, x.y, v.z, v.w);
              df_mac(wih, wil, x.z, x.w, v.x, v.y);
            }
            // t = tau w (double-float products, normalised)
            float trh = 0.f, trl = 0.f, tih = 0.f, til = 0.f;
            df_mac(trh, trl, tauf.x, tauf.y, wrh, wrl);
            df_mac(tih, til, tauf.x, tauf.y, wih, wil);
            // base(slot) -= t conj(v(slot))
            for (int q = 0; q <= m; ++q) {
              const int slot = q < m ? q : fs;
              float4 x = base[slot * stride];
              const float4 v = vf[slot];
              float xrh = x.x, xrl = x.y, xih = x.z, xil = x.w;
              df_mac(xrh, xrl, -trh, -trl, v.x, v.y);
              df_mac(xrh, xrl, -tih, -til, v.z, v.w);
              df_mac(xih, xil, -tih, -til, v.x, v.y);
              df_mac(xih, xil, trh, trl, v.z, v.w);
              float sr = xrh + xrl, si = xih + xil;
              x = make_float4(sr, xrl - (sr - xrh), si, xil - (si - xih));
              base[slot * stride] = x;
            }
          }
        }
        if (c > 0) {
          const int cn = c - 1;
          if (tid <= cn) cand4[fn * kNB + tid] = pre;
          for (int crow = tid; crow < L::kCoefRows; crow += kThreads)
            coef4[crow * S + fn] = make_float4(crow == cn ? 1.f : 0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
      }
    } else {
      // stage the live rows of the block and reset coefficients
      for (int idx = tid; idx < m * nbe; idx += kThreads) {
        int t = idx % nbe, q = idx / nbe;
        cand[q * kNB + t] = Z2[(r + t) + (size_t)q * ldz];
      }
      if (RHS) {
        for (int t = tid; t < nbe; t += kThreads) rhs_s[t] = Zr[r + t];
        for (int crow = tid; crow < L::kCoefRows; crow += kThreads) coefr[crow] = mkcd(0.0, 0.0);
      }
      // coefficients: identity on the old live columns, e_{nbe-1} for the
      // fresh column F_{nbe-1} that enters slot m (slots m, m+1 alternate)
      for (int idx = tid; idx < L::kCoefRows * S; idx += kThreads) {
        int c = idx / S, slot = idx % S;
        cd v = mkcd(0.0, 0.0);
        if ((slot < m && c == kNB + slot) || (slot == m && c == nbe - 1)) v = mkcd(1.0, 0.0);
        coef[idx] = v;
      }
      {
        const int c = nbe - 1, jc = j0 + c;
        for (int t = tid; t <= c; t += kThreads) {
          cd z = mkcd(H[(k - nbe + t) + (size_t)jc * n], 0.0);
          if (t == c - m) z = csub(z, sigma);
          cand[m * kNB + t] = z;
        }
      }
      __syncthreads();
      for (int c = nbe - 1; c >= 0; --c) {
        const int fs = m + ((nbe - 1 - c) & 1);  // slot holding F_c
        const int fn = (fs == m) ? m + 1 : m;    // slot for F_{c-1}
        // ---- reflector U = I - tau v v^H on the m + 1 candidates of row c
        //      (survivors 0..m-1, fresh fs): x U = conj(alpha) e_fs, x = row c.
        if (tid < 32) {
          double rest2 = 0.0;  // sum of |x_q|^2 over the m survivors
          for (int q = tid; q < m; q += 32) {
            const cd x = cand[q * kNB + c];
            rest2 = fma(x.x, x.x, fma(x.y, x.y, rest2));
          }
          for (int o = 16; o > 0; o >>= 1) rest2 += __shfl_xor_sync(0xffffffffu, rest2, o);
          const cd xf = cand[fs * kNB + c];
          const double af2 = fma(xf.x, xf.x, xf.y * xf.y);
          const double af = sqrt(af2);
          const double nrm2 = rest2 + af2;
          const double nrm = sqrt(nrm2);
          // y = conj(x); alpha = -exp(i arg y_fs) ||y||; v = y - alpha e_fs
          cd ph = af > 0.0 ? mkcd(xf.x / af, -xf.y / af) : mkcd(1.0, 0.0);
          const cd alpha = mkcd(-ph.x * nrm, -ph.y * nrm);
          const bool trivial = !(rest2 > 0.0);
          for (int q = tid; q <= m; q += 32) {
            const int slot = q < m ? q : fs;
            const cd x = cand[slot * kNB + c];
            cd v = mkcd(x.x, -x.y);
            if (slot == fs) v = csub(v, alpha);
            lmul[slot] = v;
          }
          if (tid == 0) {
            // ||v||^2 = 2 ||y||^2 + 2 |y_fs| ||y||
            const double vv = 2.0 * nrm2 + 2.0 * af * nrm;
            lmul[MAXM + 2].x = trivial ? 0.0 : 2.0 / vv;
            // finalised diagonal entry of row c: conj(alpha) (x_fs when no reflection)
            lmul[MAXM + 3] = trivial ? xf : mkcd(alpha.x, -alpha.y);
            if (nrm <= sing_tol) s_sing = 1;  // |R(row, row)| = ||x|| at working precision
          }
        }
        __syncthreads();
        const double tau = lmul[MAXM + 2].x;
        // ---- apply to window rows 0..c-1 and the nonzero coefficient rows;
        //      load F_{c-1} into slot fn meanwhile.
        if (tau != 0.0) {
          const int nrow = c;
          const int ncoef = (nbe - c) + m;
          for (int e = tid; e < nrow + ncoef; e += kThreads) {
            cd* base;
            int stride;
            if (e < nrow) {
              base = cand + e;
              stride = kNB;
            } else {
              const int ee = e - nrow;
              const int crow = ee < nbe - c ? c + ee : kNB + (ee - (nbe - c));
              base = coef + crow * S;
              stride = 1;
            }
            cd w = mkcd(0.0, 0.0);
            for (int q = 0; q <= m; ++q) {
              const int slot = q < m ? q : fs;
              w = cfma(base[slot * stride], lmul[slot], w);
            }
            w = mkcd(w.x * tau, w.y * tau);
            for (int q = 0; q <= m; ++q) {
              const int slot = q < m ? q : fs;
              const cd vc = mkcd(lmul[slot].x, -lmul[slot].y);
              base[slot * stride] = cfms(w, vc, base[slot * stride]);
            }
          }
        }
        if (RHS) {
          // back substitution with the finalised column F_c (slot fs)
          __syncthreads();
          const cd beta = lmul[MAXM + 3];
          const cd f = (beta.x == 0.0 && beta.y == 0.0) ? mkcd(0.0, 0.0) : cdiv(rhs_s[c], beta);
          const int nrow = c;
          const int ncoef = (nbe - c) + m;
          for (int e = tid; e < nrow + ncoef; e += kThreads) {
            if (e < nrow) {
              rhs_s[e] = cfms(f, cand[fs * kNB + e], rhs_s[e]);
            } else {
              const int ee = e - nrow;
              const int crow = ee < nbe - c ? c + ee : kNB + (ee - (nbe - c));
              coefr[crow] = cfms(f, coef[crow * S + fs], coefr[crow]);
            }
          }
        }
        if (c > 0) {
          const int cn = c - 1, jc = j0 + cn;
          for (int t = tid; t <= cn; t += kThreads) {
            cd z = mkcd(H[(k - nbe + t) + (size_t)jc * n], 0.0);
            if (t == cn - m) z = csub(z, sigma);
            cand[fn * kNB + t] = z;
          }
          for (int crow = tid; crow < L::kCoefRows; crow += kThreads)
            coef[crow * S + fn] = mkcd(crow == cn ? 1.0 : 0.0, 0.0);
        }
        __syncthreads();
      }
    }

    // ---- update the rows above the block (and the T rows)
    if constexpr (DF) {
      // double-float update (SSV_DFLOAT): the coefficients as FP32 pairs
      // (re_hi, re_lo, im_hi, im_lo), H as (Hhi, Hlo), Z2 split on the
      // fly; exact FMA products, two-sum accumulation (48-bit class).  The Ct
      // rows and the diagonal correction stay in FP64.
      // (the double-float panel above left `coef` in this form already)
      static_assert(!(DF && (GIVENS || RHS)), "double-float updates need the double-float panel");
    }
    auto coefd = [&](int crow, int q) -> cd {
      if constexpr (DF) {
        const float4 w = reinterpret_cast<const float4*>(coef)[crow * S + q];
        return mkcd((double)w.x + (double)w.y, (double)w.z + (double)w.w);
      } else {
        return coef[crow * S + q];
      }
    };
    if constexpr (DF) {
      const float4* cf4 = reinterpret_cast<const float4*>(coef);
      for (int i = tid; i < r; i += kThreads) {
        cd acc[MAXM];
        if (i < p) {
#pragma unroll
          for (int q = 0; q < MAXM; ++q) acc[q] = mkcd(0.0, 0.0);
          for (int c = 0; c < nbe; ++c) {
            const double z = Ct[i + (size_t)(j0 + c) * ldct];
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
              if (q < m) {
                const cd w = coefd(c, q);
                acc[q].x = fma(z, w.x, acc[q].x);
                acc[q].y = fma(z, w.y, acc[q].y);
              }
            }
          }
          for (int qq = 0; qq < m; ++qq) {
            const cd zz = df_join(Z2f[i + (size_t)qq * ldz]);
#pragma unroll
            for (int q = 0; q < MAXM; ++q)
              if (q < m) acc[q] = cfma(zz, coefd(LB + qq, q), acc[q]);
          }
        } else {
          float rh[MAXM], rl[MAXM], ih[MAXM], il[MAXM];
#pragma unroll
          for (int q = 0; q < MAXM; ++q) { rh[q] = 0.f; rl[q] = 0.f; ih[q] = 0.f; il[q] = 0.f; }
          const size_t row = (size_t)(i - p);
          for (int c = 0; c < nbe; ++c) {
            const size_t hidx = row + (size_t)(j0 + c) * n;
            const float zh = d.Hhi[hidx], zl = d.Hlo[hidx];
            const float4* cr = cf4 + c * S;
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
              if (q < m) {
                const float4 w = cr[q];
                df_mac(rh[q], rl[q], zh, zl, w.x, w.y);
                df_mac(ih[q], il[q], zh, zl, w.z, w.w);
              }
            }
          }
          for (int qq = 0; qq < m; ++qq) {
            const float4 zz = Z2f[i + (size_t)qq * ldz];
            const float zrh = zz.x, zrl = zz.y, zih = zz.z, zil = zz.w;
            const float4* cr = cf4 + (LB + qq) * S;
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
              if (q < m) {
                const float4 w = cr[q];
                // (zr + i zi)(wr + i wi) = (zr wr - zi wi) + i (zr wi + zi wr)
                df_mac(rh[q], rl[q], zrh, zrl, w.x, w.y);
                df_mac(rh[q], rl[q], -zih, -zil, w.z, w.w);
                df_mac(ih[q], il[q], zrh, zrl, w.z, w.w);
                df_mac(ih[q], il[q], zih, zil, w.x, w.y);
              }
            }
          }
          const int cd_ = i - (r - m);  // diagonal correction of fresh column cd_
          if (!(cd_ >= 0 && cd_ < min(m, nbe))) {
            // normalised pairs straight back into the window state
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
              if (q < m) {
                const float sr = rh[q] + rl[q], si = ih[q] + il[q];
                Z2f[i + (size_t)q * ldz] =
                    make_float4(sr, rl[q] - (sr - rh[q]), si, il[q] - (si - ih[q]));
              }
            }
            continue;
          }
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            acc[q] = mkcd((double)rh[q] + (double)rl[q], (double)ih[q] + (double)il[q]);
        }
        const int cd_ = i - (r - m);  // diagonal correction of fresh column cd_
        if (cd_ >= 0 && cd_ < min(m, nbe)) {
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            if (q < m) acc[q] = cfms(sigma, coefd(cd_, q), acc[q]);
        }
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) z2st(i + (size_t)q * ldz, acc[q]);
      }
    } else
    for (int i = tid; i < r; i += kThreads) {
      cd acc[MAXM];
      cd racc = mkcd(0.0, 0.0);
      if (RHS) racc = Zr[i];
#pragma unroll
      for (int q = 0; q < MAXM; ++q) acc[q] = mkcd(0.0, 0.0);
      for (int c = 0; c < nbe; ++c) {
        const int jc = j0 + c;
        const double z = i < p ? Ct[i + (size_t)jc * ldct] : H[(i - p) + (size_t)jc * n];
        const cd* cr = coef + c * S;
#pragma unroll
        for (int q = 0; q < MAXM; ++q) {
          if (q < m) {
            cd w = cr[q];
            acc[q].x = fma(z, w.x, acc[q].x);
            acc[q].y = fma(z, w.y, acc[q].y);
          }
        }
        if (RHS) racc = mkcd(fma(z, coefr[c].x, racc.x), fma(z, coefr[c].y, racc.y));
      }
      for (int qq = 0; qq < m; ++qq) {
        const cd zz = Z2[i + (size_t)qq * ldz];
        const cd* cr = coef + (LB + qq) * S;
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) acc[q] = cfma(zz, cr[q], acc[q]);
        if (RHS) racc = cfma(zz, coefr[kNB + qq], racc);
      }
      const int cd_ = i - (r - m);  // diagonal correction of fresh column cd_
      if (cd_ >= 0 && cd_ < min(m, nbe)) {
        const cd* cr = coef + cd_ * S;
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) acc[q] = cfms(sigma, cr[q], acc[q]);
        if (RHS) racc = cfms(sigma, coefr[cd_], racc);
      }
      if (RHS) Zr[i] = racc;
#pragma unroll
      for (int q = 0; q < MAXM; ++q)
        if (q < m) Z2[i + (size_t)q * ldz] = acc[q];
    }
    if (defer_t) {
      // rows j0 .. j0+nbe-1: ZT = P1; P2 parked in the output (see above)
      for (int idx = tid; idx < nbe * m; idx += kThreads) {
        const int i = j0 + idx % nbe, q = idx / nbe;
        ZT[i + (size_t)q * n] = coefd(i - j0, q);
      }
      for (int idx = tid; idx < m * m; idx += kThreads) {
        const int qq = idx % m, q = idx / m;
        tout[(n - nsteps * m + qq) + (size_t)q * tld] = coefd(LB + qq, q);
      }
    } else if (track_t) {
      // rows k-m .. n-1: ZT <- ZT P2 ; rows j0 .. j0+nbe-1: ZT = P1
      const int lo = k - m;
      for (int i = j0 + tid; i < n; i += kThreads) {
        cd acc[MAXM];
        if (RHS) {
          cd tr;
          if (i < lo) {
            tr = coefr[i - j0];
          } else {
            tr = Tr[i];
            for (int qq = 0; qq < m; ++qq) tr = cfma(ZT[i + (size_t)qq * n], coefr[kNB + qq], tr);
          }
          Tr[i] = tr;
        }
        if (i < lo) {
#pragma unroll
          for (int q = 0; q < MAXM; ++q) acc[q] = coefd(i - j0, q);
        } else if constexpr (DF) {
          float rh[MAXM], rl[MAXM], ih[MAXM], il[MAXM];
#pragma unroll
          for (int q = 0; q < MAXM; ++q) { rh[q] = 0.f; rl[q] = 0.f; ih[q] = 0.f; il[q] = 0.f; }
          for (int qq = 0; qq < m; ++qq) {
            const cd zz = ZT[i + (size_t)qq * n];
            const float zrh = (float)zz.x, zrl = (float)(zz.x - (double)zrh);
            const float zih = (float)zz.y, zil = (float)(zz.y - (double)zih);
            const float4* cr = reinterpret_cast<const float4*>(coef) + (LB + qq) * S;
#pragma unroll
            for (int q = 0; q < MAXM; ++q) {
              if (q < m) {
                const float4 w = cr[q];
                df_mac(rh[q], rl[q], zrh, zrl, w.x, w.y);
                df_mac(rh[q], rl[q], -zih, -zil, w.z, w.w);
                df_mac(ih[q], il[q], zrh, zrl, w.z, w.w);
                df_mac(ih[q], il[q], zih, zil, w.x, w.y);
              }
            }
          }
#pragma unroll
          for (int q = 0; q < MAXM; ++q)
            acc[q] = mkcd((double)rh[q] + (double)rl[q], (double)ih[q] + (double)il[q]);
        } else {
#pragma unroll
          for (int q = 0; q < MAXM; ++q) acc[q] = mkcd(0.0, 0.0);
          for (int qq = 0; qq < m; ++qq) {
            const cd zz = ZT[i + (size_t)qq * n];
#pragma unroll
            for (int q = 0; q < MAXM; ++q)
              if (q < m) acc[q] = cfma(zz, coefd(LB + qq, q), acc[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
          if (q < m) ZT[i + (size_t)q * n] = acc[q];
      }
    }
    __syncthreads();
    k -= nbe;
  }

  // ---- final m x m block: solve Wm Y = R(0:m, 0:m) by Gauss-Jordan with
  // partial pivoting on the augmented [Wm | R1] (2m columns).  With a
  // right-hand side per shift (Sec. 3.3) the augmented part is the single
  // column R1 bhat, and Y is m x 1.
  const cd* __restrict__ bh = d.bhat != nullptr ? d.bhat + (size_t)sh * d.ldb : nullptr;
  const int nr = (RHS || bh != nullptr) ? 1 : m;
  const int w2 = m + nr;
  for (int idx = tid; idx < m * w2; idx += kThreads) {
    int i = idx % m, j = idx / m;
    cd v;
    if (j < m) v = z2ld((p + i) + (size_t)j * ldz);
    else if (RHS) {
      v = Zr[i];
    } else if (bh != nullptr) {
      v = mkcd(0.0, 0.0);
      for (int t = i; t < m; ++t) {
        const double rv = R[i + (size_t)t * n];
        v = mkcd(fma(rv, bh[t].x, v.x), fma(rv, bh[t].y, v.y));
      }
    } else {
      int jj = j - m;
      v = mkcd(i <= jj ? R[i + (size_t)jj * n] : 0.0, 0.0);
    }
    Wm[i + j * MAXM] = v;
  }
  __syncthreads();
  for (int kk = 0; kk < m; ++kk) {
    if (tid < 32) {
      double best = -1.0;
      int brow = kk;
      for (int i = kk + tid; i < m; i += 32) {
        double v = cabs1(Wm[i + kk * MAXM]);
        if (v > best) { best = v; brow = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int orow = __shfl_xor_sync(0xffffffffu, brow, o);
        if (ob > best || (ob == best && orow < brow)) { best = ob; brow = orow; }
      }
      if (tid == 0) {
        s_piv = brow;
        const cd pv = Wm[brow + kk * MAXM];
        if (best == 0.0 || sqrt(pv.x * pv.x + pv.y * pv.y) <= sing_tol) s_sing = 1;
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != kk) {
      for (int j = tid; j < w2; j += kThreads) {
        cd a = Wm[kk + j * MAXM];
        Wm[kk + j * MAXM] = Wm[pr + j * MAXM];
        Wm[pr + j * MAXM] = a;
      }
    }
    __syncthreads();
    const cd d = Wm[kk + kk * MAXM];
    const bool dz = (d.x == 0.0 && d.y == 0.0);
    if (tid < m) lmul[tid] = (tid == kk || dz) ? mkcd(0.0, 0.0) : cdiv(Wm[tid + kk * MAXM], d);
    __syncthreads();
    for (int idx = tid; idx < m * w2; idx += kThreads) {
      int i = idx % m, j = idx / m;
      if (i != kk && j > kk) Wm[i + j * MAXM] = cfms(lmul[i], Wm[kk + j * MAXM], Wm[i + j * MAXM]);
    }
    __syncthreads();
  }
  // Y(i, q) = Wm(i, m+q) / Wm(i, i)
  for (int idx = tid; idx < m * nr; idx += kThreads) {
    int i = idx % m, q = idx / m;
    cd d = Wm[i + i * MAXM];
    Yb[i + q * MAXM] = (d.x == 0.0 && d.y == 0.0) ? mkcd(0.0, 0.0) : cdiv(Wm[i + (m + q) * MAXM], d);
  }
  __syncthreads();
  const bool sing = s_sing != 0;
  const double nanv = __longlong_as_double(0x7ff8000000000000LL);
  // ---- outputs
  if (mode == SSV_G || mode == SSV_TF) {
    const double sg = mode == SSV_TF ? -1.0 : 1.0;
    cd* o = out + (size_t)sh * nr * ldo;
    for (int idx = tid; idx < p * nr; idx += kThreads) {
      int i = idx % p, q = idx / p;
      cd acc = mkcd(0.0, 0.0);
      for (int t = 0; t < m; ++t) acc = cfma(z2ld(i + (size_t)t * ldz), Yb[t + q * MAXM], acc);
      if (sing) acc = mkcd(nanv, nanv);
      o[i + (size_t)q * ldo] = mkcd(sg * acc.x, sg * acc.y);
    }
  }
  if (defer_t) {
    // backward pass: z = Y; per step b = B .. 1: X-hat rows of b = P1_b z,
    // then z = P2_b z; finally the initial live rows n-m .. n-1 take z
    cd* zs = cand;                // m x m (ld MAXM)
    cd* p2s = zs + MAXM * MAXM;   // P2_b
    cd* zn = p2s + MAXM * MAXM;   // P2_b z
    static_assert(L::cand_elems >= 3 * MAXM * MAXM, "backward-pass scratch");
    for (int e = tid; e < m * m; e += kThreads) zs[(e % m) + (e / m) * MAXM] = Yb[(e % m) + (e / m) * MAXM];
    __syncthreads();
    for (int b = nsteps; b >= 1; --b) {
      const int kb = n - (b - 1) * nb;  // every step before the last takes nb rows
      const int nbe_b = min(nb, kb - m);
      const int j0b = kb - m - nbe_b;
      for (int e = tid; e < m * m; e += kThreads)
        p2s[(e % m) + (e / m) * MAXM] = tout[(n - b * m + e % m) + (size_t)(e / m) * tld];
      __syncthreads();
      for (int idx = tid; idx < nbe_b * m; idx += kThreads) {
        const int i = j0b + idx % nbe_b, q = idx / nbe_b;
        cd acc = mkcd(0.0, 0.0);
        for (int t = 0; t < m; ++t) acc = cfma(ZT[i + (size_t)t * n], zs[t + q * MAXM], acc);
        tout[i + (size_t)q * tld] = sing ? mkcd(nanv, nanv) : acc;
      }
      for (int e = tid; e < m * m; e += kThreads) {
        const int rr = e % m, q = e / m;
        cd acc = mkcd(0.0, 0.0);
        for (int t = 0; t < m; ++t) acc = cfma(p2s[rr + t * MAXM], zs[t + q * MAXM], acc);
        zn[rr + q * MAXM] = acc;
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += kThreads) zs[(e % m) + (e / m) * MAXM] = zn[(e % m) + (e / m) * MAXM];
      __syncthreads();
    }
    for (int e = tid; e < m * m; e += kThreads) {
      const int rr = e % m, q = e / m;
      tout[(n - m + rr) + (size_t)q * tld] = sing ? mkcd(nanv, nanv) : zs[rr + q * MAXM];
    }
  } else if (track_t) {
    cd* o;
    long long ld;
    if (mode == SSV_XHAT || mode == SSV_X) {
      o = out + (size_t)sh * nr * ldo;
      ld = ldo;
    } else {
      o = xhat_copy + (size_t)sh * nr * ldxc;
      ld = ldxc;
    }
    for (int idx = tid; idx < n * nr; idx += kThreads) {
      int i = idx % n, q = idx / n;
      cd acc = mkcd(0.0, 0.0);
      if (RHS) acc = mkcd(-Tr[i].x, -Tr[i].y);
      for (int t = 0; t < m; ++t) acc = cfma(ZT[i + (size_t)t * n], Yb[t + q * MAXM], acc);
      if (sing) acc = mkcd(nanv, nanv);
      o[(d.flip_out ? n - 1 - i : i) + (size_t)q * ld] = acc;
    }
  }
  if (status != nullptr && tid == 0) {
    // a non-finite solution (NaN / Inf in the inputs or an overflow) is reported
    // as such, also when no separate scan of the outputs follows
    bool fin = true;
    for (int e = 0; e < m * nr; ++e) {
      const cd y = Yb[(e % m) + (e / m) * MAXM];
      fin = fin && isfinite(y.x) && isfinite(y.y);
    }
    status[sh] = sing ? SSV_SHIFT_SINGULAR : (fin ? SSV_SHIFT_OK : SSV_SHIFT_NONFINITE);
  }
  __syncthreads();
}

template <int MAXM, bool DF = false>
__global__ void __launch_bounds__(kThreads, MAXM <= 16 ? 2 : 1) solve_fp64_kernel(
    int n, int m, int p, int nb, const double* __restrict__ H, const double* __restrict__ Ct,
    int ldct, const double* __restrict__ R, int s, const cd* __restrict__ shifts, int mode,
    cd* __restrict__ scratch, size_t slot_stride, cd* __restrict__ out, long long ldo,
    int* __restrict__ status, cd* __restrict__ xhat_copy, long long ldxc,
    const double* __restrict__ hnorm, const int* __restrict__ list,
    const int* __restrict__ count, const cd* __restrict__ bhat, long long ldb,
    const float* __restrict__ Hhi, const float* __restrict__ Hlo) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_piv;
  __shared__ int s_sing;
  FpSys d;
  d.n = n; d.m = m; d.p = p; d.nb = nb; d.mode = mode; d.H = H; d.Ct = Ct; d.ldct = ldct;
  d.R = R; d.shifts = shifts; d.out = out; d.ldo = ldo; d.status = status;
  d.xhat_copy = xhat_copy; d.ldxc = ldxc; d.hnorm = hnorm; d.bhat = bhat; d.ldb = ldb;
  d.rhs = nullptr; d.ldr = 0; d.flip_out = 0;
  d.Hhi = Hhi; d.Hlo = Hlo;
  d.gfull = GivensSched{nullptr, nullptr, 0};
  d.gtail = d.gfull;
  cd* Z2 = scratch + (size_t)blockIdx.x * slot_stride;
  // With a work list, the block takes list entries blockIdx.x, +gridDim.x, ...
  const int nwork = list != nullptr ? *count : s;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int sh = list != nullptr ? list[w] : w;
    fp64_shift<MAXM, false, false, DF>(d, sh, Z2, smem_raw, &s_piv, &s_sing);
  }
}

// Givens-panel sweep (Sec. 3.2): the same work list as solve_fp64_kernel.
template <int MAXM>
__global__ void __launch_bounds__(kThreads) solve_fp64_givens_kernel(FpSys d, int s,
                                                                     cd* __restrict__ scratch,
                                                                     size_t slot_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_piv;
  __shared__ int s_sing;
  cd* Z2 = scratch + (size_t)blockIdx.x * slot_stride;
  for (int w = blockIdx.x; w < s; w += gridDim.x)
    fp64_shift<MAXM, false, true>(d, w, Z2, smem_raw, &s_piv, &s_sing);
}

// Dense right-hand side per shift (the transposed systems of Sec. 3.3, in the
// flipped form built by solve_fp64_trans); d.p == 0.
template <int MAXM>
__global__ void __launch_bounds__(kThreads) solve_fp64_rhs_kernel(FpSys d, int s,
                                                                  cd* __restrict__ scratch,
                                                                  size_t slot_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_piv;
  __shared__ int s_sing;
  cd* Z2 = scratch + (size_t)blockIdx.x * slot_stride;
  for (int w = blockIdx.x; w < s; w += gridDim.x)
    fp64_shift<MAXM, true>(d, w, Z2, smem_raw, &s_piv, &s_sing);
}

// Ht(i, j) = H(n-1-j, n-1-i) on the structural part i <= j + m, zero below:
// J (H - sigma I)^T J = Ht - sigma I is upper m-Hessenberg again.  32 x 32
// tiles through shared memory, coalesced on both sides.
__global__ void flip_transpose_kernel(const double* __restrict__ H, int n, int m,
                                      double* __restrict__ Ht) {
  __shared__ double tile[32][33];
  const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;  // rows / columns of H
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int k = 0; k < 32; k += 8) {
    const int a = a0 + tx, b = b0 + ty + k;
    tile[ty + k][tx] = (a < n && b < n) ? H[a + (size_t)b * n] : 0.0;
  }
  __syncthreads();
  for (int k = 0; k < 32; k += 8) {
    const int b = b0 + tx, a = a0 + ty + k;
    if (a < n && b < n) {
      const int i = n - 1 - b, j = n - 1 - a;
      Ht[i + (size_t)j * n] = (i <= j + m) ? tile[tx][ty + k] : 0.0;
    }
  }
}

// d(i, l) = (Ct^T chat_l)(n-1-i): the flipped reduced right-hand side C~^T chat_l.
__global__ void flipped_rhs_kernel(const double* __restrict__ Ct, int ldct, int p, int n,
                                   const cd* __restrict__ chat, long long ldc, int s,
                                   cd* __restrict__ dvec) {
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < (long long)n * s;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % n), l = (int)(idx / n);
    const int col = n - 1 - i;
    const cd* c = chat + (size_t)l * ldc;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < p; ++k) {
      const double v = Ct[k + (size_t)col * ldct];
      re = fma(v, c[k].x, re);
      im = fma(v, c[k].y, im);
    }
    dvec[idx] = mkcd(re, im);
  }
}

// Many systems in one launch: work item w = (system, shift) from `items`
// (system in the high 32 bits), ordered by decreasing cost.
template <int MAXM, bool DF = false>
__global__ void __launch_bounds__(kThreads, MAXM <= 16 ? 2 : 1) solve_fp64_batch_kernel(
    const FpSys* __restrict__ systems, const unsigned long long* __restrict__ items, int nitems,
    cd* __restrict__ scratch, size_t slot_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_piv;
  __shared__ int s_sing;
  cd* Z2 = scratch + (size_t)blockIdx.x * slot_stride;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const unsigned long long it = items[w];
    const FpSys d = systems[(int)(it >> 32)];
    fp64_shift<MAXM, false, false, DF>(d, (int)(it & 0xffffffffu), Z2, smem_raw, &s_piv, &s_sing);
  }
}

// Non-finite scan: status[sh] = NONFINITE if an output of an OK shift is not finite.
__global__ void nonfinite_kernel(const cd* __restrict__ out, long long ldo, int rows, int m, int s,
                                 int* __restrict__ status) {
  int sh = blockIdx.x;
  if (sh >= s) return;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  const cd* o = out + (size_t)sh * m * ldo;
  for (int idx = threadIdx.x; idx < rows * m; idx += blockDim.x) {
    int i = idx % rows, q = idx / rows;
    cd v = o[i + (size_t)q * ldo];
    if (!isfinite(v.x) || !isfinite(v.y)) bad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0 && bad && status[sh] == SSV_SHIFT_OK) status[sh] = SSV_SHIFT_NONFINITE;
}

template <int MAXM, bool DF = false>
int launch_solve(const Handle* h, int s, const double* shifts, int nb, int mode, double* out,
                 long long ldo, int* status, cd* xhat_copy, long long ldxc, cudaStream_t st,
                 const int* list = nullptr, const int* count = nullptr,
                 const cd* bhat = nullptr, long long ldb = 0) {
  using L = Layout<MAXM>;
  const int n = h->n, m = h->m, p = h->p;
  const bool track_t = (mode == SSV_XHAT || mode == SSV_X || xhat_copy != nullptr);
  const size_t slot = (size_t)(p + n) * m + (track_t ? (size_t)n * m : 0);
  int dev = 0;
  SSV_CUDA_TRY(cudaGetDevice(&dev));
  auto kern = solve_fp64_kernel<MAXM, DF>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
  int per_sm = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L::bytes));
  per_sm = std::max(1, std::min(per_sm, 2));
  int grid = std::min(s, num_sms() * per_sm);
  cd* scratch = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&scratch, sizeof(cd) * slot * grid, st));
  kern<<<grid, kThreads, L::bytes, st>>>(n, m, p, nb, h->H, h->Ct, p > 0 ? p : 1, h->R, s,
                                         reinterpret_cast<const cd*>(shifts), mode, scratch, slot,
                                         reinterpret_cast<cd*>(out), ldo, status, xhat_copy, ldxc,
                                         h->hnorm2, list, count, bhat, ldb, h->Hhi, h->Hlo);
  count_launch();
  cudaError_t e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    set_cuda_error(e);
    return SSV_ECUDA;
  }
  if (status != nullptr && list == nullptr) {
    int rows = (mode == SSV_G || mode == SSV_TF) ? p : n;
    if (rows > 0) {
      nonfinite_kernel<<<s, 256, 0, st>>>(reinterpret_cast<const cd*>(out), ldo, rows,
                                          bhat != nullptr ? 1 : m, s, status);
      count_launch();
      SSV_CUDA_TRY(cudaGetLastError());
    }
  }
  return SSV_OK;
}

}  // namespace

// Default block width of the FP64 sweep: n_b = 128 halves the per-shift
// Z2 P2 work of n_b = 64 at the price of a longer panel (measured 9 % faster
// at n = 5000, m = 16); small problems keep 64.
int default_nb(int n, int m) {
  (void)m;
  return n >= 1024 ? 128 : 64;
}

// Work list of the shifts with mask[j] != 0 (single block, order preserved).
__global__ void __launch_bounds__(1024) mask_to_list_kernel(int s, const int* __restrict__ mask,
                                                            int* __restrict__ list,
                                                            int* __restrict__ count) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int chunk = (s + 1023) / 1024;
  const int b = tid * chunk, e = min(s, b + chunk);
  int c = 0;
  for (int j = b; j < e; ++j) c += mask[j] != 0;
  part[tid] = c;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v = tid >= o ? part[tid - o] : 0;
    __syncthreads();
    part[tid] += v;
    __syncthreads();
  }
  int pos = part[tid] - c;
  for (int j = b; j < e; ++j)
    if (mask[j] != 0) list[pos++] = j;
  if (tid == 1023) *count = part[1023];
}

int solve_fp64_masked(const Handle* h, int s, const double* shifts, int mode, int nb,
                      double* out, long long ldo, int* status, const int* mask, void* xhat_copy,
                      long long ldxc, cudaStream_t st) {
  const int m = h->m;
  if (nb <= 0) nb = default_nb(h->n, m);
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  int* list = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&list, sizeof(int) * ((size_t)s + 1), st));
  int* count = list + s;
  mask_to_list_kernel<<<1, 1024, 0, st>>>(s, mask, list, count);
  count_launch();
  cd* xc = reinterpret_cast<cd*>(xhat_copy);
  int rc;
  if (m <= 1) rc = launch_solve<1>(h, s, shifts, nb, mode, out, ldo, status, xc, ldxc, st, list, count);
  else if (m <= 2) rc = launch_solve<2>(h, s, shifts, nb, mode, out, ldo, status, xc, ldxc, st, list, count);
  else if (m <= 4) rc = launch_solve<4>(h, s, shifts, nb, mode, out, ldo, status, xc, ldxc, st, list, count);
  else if (m <= 8) rc = launch_solve<8>(h, s, shifts, nb, mode, out, ldo, status, xc, ldxc, st, list, count);
  else if (m <= 16) rc = launch_solve<16>(h, s, shifts, nb, mode, out, ldo, status, xc, ldxc, st, list, count);
  else if (m <= 32) rc = launch_solve<32>(h, s, shifts, nb, mode, out, ldo, status, xc, ldxc, st, list, count);
  else rc = SSV_ENOTSUP;
  cudaError_t e = cudaFreeAsync(list, st);
  if (e != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e);
    rc = SSV_ECUDA;
  }
  return rc;
}

size_t solve_fp64_scratch_bytes(int n, int m, int p, int s, const ssv_opts* o) {
  const bool track_t = (o->mode == SSV_XHAT || o->mode == SSV_X);
  size_t slot = (size_t)(p + n) * m + (track_t ? (size_t)n * m : 0);
  size_t grid = (size_t)std::min(s, num_sms() * 2);
  return sizeof(cd) * slot * grid + 256;
}

int solve_fp64(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
               long long ldo, int* status, double* resid, cudaStream_t st) {
  const int m = h->m;
  int nb = o->nb > 0 ? o->nb : tuned_nb(h->n, m, h->p, o->precision, o->mode);
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  cd* xcopy = nullptr;
  long long ldxc = 0;
  if (resid != nullptr && (o->mode == SSV_G || o->mode == SSV_TF)) {
    ldxc = h->n;
    SSV_CUDA_TRY(pool_alloc((void**)&xcopy, sizeof(cd) * (size_t)h->n * m * s, st));
  }
  int rc;
  if (o->precision == SSV_DFLOAT) {
    if (m <= 1) rc = launch_solve<1, true>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 2) rc = launch_solve<2, true>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 4) rc = launch_solve<4, true>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 8) rc = launch_solve<8, true>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 16) rc = launch_solve<16, true>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 32) rc = launch_solve<32, true>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else rc = SSV_ENOTSUP;
  } else {
    if (m <= 1) rc = launch_solve<1>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 2) rc = launch_solve<2>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 4) rc = launch_solve<4>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 8) rc = launch_solve<8>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 16) rc = launch_solve<16>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else if (m <= 32) rc = launch_solve<32>(h, s, shifts, nb, o->mode, out, ldo, status, xcopy, ldxc, st);
    else rc = SSV_ENOTSUP;
  }
  if (rc == SSV_OK && resid != nullptr) {
    const double* xh = xcopy ? reinterpret_cast<const double*>(xcopy) : out;
    long long ldx = xcopy ? ldxc : ldo;
    rc = backward_error_fp64(h, s, shifts, xh, ldx, resid, st);
  }
  if (xcopy) {
    cudaError_t e = cudaFreeAsync(xcopy, st);
    if (e != cudaSuccess && rc == SSV_OK) {
      set_cuda_error(e);
      rc = SSV_ECUDA;
    }
  }
  return rc;
}

// One right-hand side B bhat_l per shift (Sec. 3.3): out column l holds
// Xhat_l bhat_l (SSV_XHAT / SSV_X before the back-transform) or
// +-Ct Xhat_l bhat_l (SSV_G / SSV_TF).
int solve_fp64_rhs(const Handle* h, int s, const double* shifts, const double* bhat,
                   long long ldb, const ssv_opts* o, double* out, long long ldo, int* status,
                   cudaStream_t st) {
  const int m = h->m;
  const int nb = o->nb > 0 ? o->nb : tuned_nb(h->n, m, h->p, SSV_FP64, o->mode);
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  const int mode = o->mode == SSV_X ? SSV_XHAT : o->mode;
  const cd* b = reinterpret_cast<const cd*>(bhat);
  if (m <= 1) return launch_solve<1>(h, s, shifts, nb, mode, out, ldo, status, nullptr, 0, st, nullptr, nullptr, b, ldb);
  if (m <= 2) return launch_solve<2>(h, s, shifts, nb, mode, out, ldo, status, nullptr, 0, st, nullptr, nullptr, b, ldb);
  if (m <= 4) return launch_solve<4>(h, s, shifts, nb, mode, out, ldo, status, nullptr, 0, st, nullptr, nullptr, b, ldb);
  if (m <= 8) return launch_solve<8>(h, s, shifts, nb, mode, out, ldo, status, nullptr, 0, st, nullptr, nullptr, b, ldb);
  if (m <= 16) return launch_solve<16>(h, s, shifts, nb, mode, out, ldo, status, nullptr, 0, st, nullptr, nullptr, b, ldb);
  if (m <= 32) return launch_solve<32>(h, s, shifts, nb, mode, out, ldo, status, nullptr, 0, st, nullptr, nullptr, b, ldb);
  return SSV_ENOTSUP;
}
namespace {
template <int MAXM>
int launch_rhs(const FpSys& d, int s, cudaStream_t st) {
  using L = Layout<MAXM>;
  const size_t slot = (size_t)d.n * d.m * 2 + 2 * (size_t)d.n;
  auto kern = solve_fp64_rhs_kernel<MAXM>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
  int per_sm = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L::bytes));
  per_sm = std::max(1, std::min(per_sm, 2));
  const int grid = std::min(s, num_sms() * per_sm);
  cd* scratch = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&scratch, sizeof(cd) * slot * grid, st));
  kern<<<grid, kThreads, L::bytes, st>>>(d, s, scratch, slot);
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

// Transposed systems (A - sigma_l I)^T x_l = C^T chat_l (Sec. 3.3) in reduced
// coordinates: (H - sigma I)^T xt = C~^T chat with x = Q xt.  With J the
// reversal, J (H - sigma I)^T J = Ht - sigma I is upper m-Hessenberg, so the
// same bottom-up sweep solves it for the dense right-hand side J C~^T chat;
// the solution is flipped back on output (out = Q^T x_l).
int solve_fp64_trans(const Handle* h, int s, const double* shifts, const double* chat,
                     long long ldc, const ssv_opts* o, double* out, long long ldo, int* status,
                     cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  const int nb = o->nb > 0 ? o->nb : tuned_nb(n, m, 0, SSV_FP64, SSV_XHAT);
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  double* Ht = nullptr;
  cd* dvec = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&Ht, sizeof(double) * (size_t)n * n, st));
  cudaError_t e = pool_alloc((void**)&dvec, sizeof(cd) * (size_t)n * s, st);
  int rc = SSV_OK;
  if (e == cudaSuccess) {
    const dim3 tg((n + 31) / 32, (n + 31) / 32);
    flip_transpose_kernel<<<tg, dim3(32, 8), 0, st>>>(h->H, n, m, Ht);
    count_launch();
    const long long tot = (long long)n * s;
    flipped_rhs_kernel<<<(int)std::min<long long>(4096, (tot + 255) / 256), 256, 0, st>>>(
        h->Ct, p > 0 ? p : 1, p, n, reinterpret_cast<const cd*>(chat), ldc, s, dvec);
    count_launch();
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    rc = e == cudaErrorMemoryAllocation ? SSV_ENOMEM : SSV_ECUDA;
  }
  if (rc == SSV_OK) {
    FpSys d;
    d.n = n; d.m = m; d.p = 0; d.nb = nb; d.mode = SSV_XHAT; d.H = Ht; d.Ct = nullptr; d.ldct = 1;
    d.R = h->R; d.shifts = reinterpret_cast<const cd*>(shifts);
    d.out = reinterpret_cast<cd*>(out); d.ldo = ldo; d.status = status;
    d.xhat_copy = nullptr; d.ldxc = 0; d.hnorm = h->hnorm2; d.bhat = nullptr; d.ldb = 0;
    d.rhs = dvec; d.ldr = n; d.flip_out = 1;
    d.gfull = GivensSched{nullptr, nullptr, 0};
    d.gtail = d.gfull;
    if (m <= 1) rc = launch_rhs<1>(d, s, st);
    else if (m <= 2) rc = launch_rhs<2>(d, s, st);
    else if (m <= 4) rc = launch_rhs<4>(d, s, st);
    else if (m <= 8) rc = launch_rhs<8>(d, s, st);
    else if (m <= 16) rc = launch_rhs<16>(d, s, st);
    else if (m <= 32) rc = launch_rhs<32>(d, s, st);
    else rc = SSV_ENOTSUP;
  }
  if (rc == SSV_OK && status != nullptr) {
    nonfinite_kernel<<<s, 256, 0, st>>>(reinterpret_cast<const cd*>(out), ldo, n, 1, s, status);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = SSV_ECUDA;
    }
  }
  if (dvec) cudaFreeAsync(dvec, st);
  if (Ht) cudaFreeAsync(Ht, st);
  return rc;
}
// ---------------------------------------------------------------------------
// Givens panel (Sec. 3.2): the greedy annihilation schedule for a block of
// `rows` rows and rows + m columns, computed on the host once per shape and
// device and kept in device memory.
//
// Row r (0-based) of the block holds nonzeros in columns r .. r + m; every
// entry but the last of a row is zeroed by a rotation with another entry of
// the same row, rotations of one step touching disjoint columns.  Seen per
// column, the entries that may be rotated form a frontier moving up: column c
// starts at its lowest band entry (row min(c, rows - 1)), and once the
// frontier entry of c is zeroed the entry above it joins in the next step;
// column c never rises above row c - m, where it survives as the diagonal of
// the triangular factor.  A step therefore looks at each row's frontier
// columns c_1 < ... < c_k and zeroes as many as the greedy choice allows:
// c_1 with the partner c_k, c_2 with c_(k-1), and so on, the middle one of an
// odd count waiting.  Steps are emitted rows from the bottom, zeroed columns
// ascending within a row, until a step finds no pair.
// ---------------------------------------------------------------------------
void greedy_rows(int rows, int m, std::vector<int>* rot, std::vector<int>* off) {
  const int cols = rows + m;
  // front[c]: row of column c's frontier entry; -1 once the column is empty
  std::vector<int> front(cols);
  for (int c = 0; c < cols; ++c) front[c] = std::min(c, rows - 1);
  std::vector<std::vector<int>> at_row(rows);
  std::vector<int> zeroed;
  rot->clear();
  off->assign(1, 0);
  for (;;) {
    for (auto& v : at_row) v.clear();
    for (int c = 0; c < cols; ++c)
      if (front[c] >= 0) at_row[front[c]].push_back(c);  // ascending in c
    zeroed.clear();
    for (int r = rows - 1; r >= 0; --r) {
      const std::vector<int>& e = at_row[r];
      const int k = (int)e.size();
      for (int i = 0; i < k / 2; ++i) {
        rot->push_back(r | (e[i] << 8) | (e[k - 1 - i] << 16));
        zeroed.push_back(e[i]);
      }
    }
    if (zeroed.empty()) break;
    for (int c : zeroed) front[c] -= 1;  // the entry above joins next step
    off->push_back((int)rot->size());
  }
}

namespace {

struct SchedEntry {
  int* rot = nullptr;
  int* off = nullptr;
  int nsteps = 0;
};
std::mutex g_sched_mu;
std::map<std::tuple<int, int, int>, SchedEntry> g_sched;  // (device, rows, m)

int givens_schedule(int rows, int m, GivensSched* out) {
  int dev = 0;
  SSV_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_sched_mu);
  auto key = std::make_tuple(dev, rows, m);
  auto it = g_sched.find(key);
  if (it == g_sched.end()) {
    std::vector<int> rot, off;
    greedy_rows(rows, m, &rot, &off);
    SchedEntry e;
    e.nsteps = (int)off.size() - 1;
    SSV_CUDA_TRY(cudaMalloc((void**)&e.rot, sizeof(int) * std::max<size_t>(1, rot.size())));
    SSV_CUDA_TRY(cudaMalloc((void**)&e.off, sizeof(int) * off.size()));
    SSV_CUDA_TRY(cudaMemcpy(e.rot, rot.data(), sizeof(int) * rot.size(), cudaMemcpyHostToDevice));
    SSV_CUDA_TRY(cudaMemcpy(e.off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    it = g_sched.emplace(key, e).first;
  }
  *out = GivensSched{it->second.rot, it->second.off, it->second.nsteps};
  return SSV_OK;
}

template <int MAXM>
int launch_givens(const FpSys& d, int s, cudaStream_t st) {
  using GL = GivensLayout<MAXM>;
  const bool track_t = (d.mode == SSV_XHAT || d.mode == SSV_X || d.xhat_copy != nullptr);
  const size_t slot = (size_t)(d.p + d.n) * d.m + (track_t ? (size_t)d.n * d.m : 0);
  auto kern = solve_fp64_givens_kernel<MAXM>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GL::bytes));
  int per_sm = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, GL::bytes));
  per_sm = std::max(1, std::min(per_sm, 2));
  const int grid = std::min(s, num_sms() * per_sm);
  cd* scratch = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&scratch, sizeof(cd) * slot * grid, st));
  kern<<<grid, kThreads, GL::bytes, st>>>(d, s, scratch, slot);
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

int solve_fp64_givens(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                      long long ldo, int* status, double* resid, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  const int nb = o->nb > 0 ? o->nb : kNBG;
  if (nb > kNBG || m > 32) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  const int mode = o->mode == SSV_X ? SSV_XHAT : o->mode;
  FpSys d;
  d.n = n; d.m = m; d.p = p; d.nb = nb; d.mode = mode; d.H = h->H; d.Ct = h->Ct;
  d.ldct = p > 0 ? p : 1; d.R = h->R; d.shifts = reinterpret_cast<const cd*>(shifts);
  d.out = reinterpret_cast<cd*>(out); d.ldo = ldo; d.status = status;
  d.xhat_copy = nullptr; d.ldxc = 0; d.hnorm = h->hnorm2; d.bhat = nullptr; d.ldb = 0;
  d.rhs = nullptr; d.ldr = 0; d.flip_out = 0;
  d.gfull = GivensSched{nullptr, nullptr, 0};
  d.gtail = d.gfull;
  const int tail = (n - m) % nb;
  int rc = SSV_OK;
  if (n > m) {
    rc = givens_schedule(std::min(nb, n - m), m, &d.gfull);
    if (rc == SSV_OK && tail != 0 && n - m > nb) rc = givens_schedule(tail, m, &d.gtail);
    if (rc == SSV_OK && n - m <= nb) d.gtail = d.gfull;
  }
  if (rc != SSV_OK) return rc;
  cd* xcopy = nullptr;
  if (resid != nullptr && (mode == SSV_G || mode == SSV_TF)) {
    SSV_CUDA_TRY(pool_alloc((void**)&xcopy, sizeof(cd) * (size_t)n * m * s, st));
    d.xhat_copy = xcopy;
    d.ldxc = n;
  }
  if (m <= 1) rc = launch_givens<1>(d, s, st);
  else if (m <= 2) rc = launch_givens<2>(d, s, st);
  else if (m <= 4) rc = launch_givens<4>(d, s, st);
  else if (m <= 8) rc = launch_givens<8>(d, s, st);
  else if (m <= 16) rc = launch_givens<16>(d, s, st);
  else rc = launch_givens<32>(d, s, st);
  if (rc == SSV_OK && status != nullptr) {
    const int rows = (mode == SSV_G || mode == SSV_TF) ? p : n;
    if (rows > 0) {
      nonfinite_kernel<<<s, 256, 0, st>>>(reinterpret_cast<const cd*>(out), ldo, rows, m, s, status);
      count_launch();
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        set_cuda_error(e);
        rc = SSV_ECUDA;
      }
    }
  }
  if (rc == SSV_OK && resid != nullptr) {
    const double* xh = xcopy ? reinterpret_cast<const double*>(xcopy) : out;
    rc = backward_error_fp64(h, s, shifts, xh, xcopy ? n : ldo, resid, st);
  }
  if (xcopy) cudaFreeAsync(xcopy, st);
  return rc;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the FP64 solve (ssv_solve_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a
// solve: code that runs while another component owns the allocator (a custom
// pool or a framework that forbids cudaMalloc / cudaMallocAsync inside its
// step), processes with a hard device-memory budget that was fixed up front,
// or real-time loops where an allocation's latency or failure is not
// acceptable.  For them the per-thread-block window state lives in one
// fixed array that is part of the loaded library image, so the call itself
// allocates nothing: no cudaMalloc / cudaMallocAsync / cudaFree and no
// allocating library routine.
//
// The array below holds kNoAllocScratchBytes (64 MiB) on every GPU where this
// translation unit's module is loaded, for as long as the process lives: any
// FP64 or double-float solve loads the module, so the 64 MiB is taken by
// those callers too, not only by callers of ssv_solve_noalloc.  In host code
// the array's name is only a host-side stand-in, so the device address is
// looked up once per device with cudaGetSymbolAddress (with that device
// current) and cached; the first call on each device performs that lookup,
// which under lazy module loading may itself load the module (an implicit
// device allocation).
// ---------------------------------------------------------------------------
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kMaxDevices = 64;
void* g_noalloc_addr[kMaxDevices] = {nullptr};

int noalloc_scratch_address(void** out) {
  int dev = 0;
  SSV_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SSV_ENOTSUP;
  if (g_noalloc_addr[dev] == nullptr) {
    void* ptr = nullptr;
    SSV_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return SSV_OK;
}

template <int MAXM>
int launch_solve_noalloc(const Handle* h, int s, const double* shifts, int nb, int mode,
                         double* out, long long ldo, int* status, cudaStream_t st) {
  using L = Layout<MAXM>;
  const int n = h->n, m = h->m, p = h->p;
  const bool track_t = (mode == SSV_XHAT);
  const size_t slot = (size_t)(p + n) * m + (track_t ? (size_t)n * m : 0);
  const size_t max_slots = kNoAllocScratchBytes / (sizeof(cd) * slot);
  if (max_slots < 1) return SSV_ESCRATCH;
  void* base = nullptr;
  int rc = noalloc_scratch_address(&base);
  if (rc != SSV_OK) return rc;
  auto kern = solve_fp64_kernel<MAXM>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
  int per_sm = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L::bytes));
  per_sm = std::max(1, std::min(per_sm, 2));
  const int grid = (int)std::min<size_t>((size_t)std::min(s, num_sms() * per_sm), max_slots);
  // Every window entry the kernel reads is written earlier in the same call
  // (the shift setup overwrites the whole slot), so nothing left in the array
  // by a previous call needs clearing.
  kern<<<grid, kThreads, L::bytes, st>>>(n, m, p, nb, h->H, h->Ct, p > 0 ? p : 1, h->R, s,
                                         reinterpret_cast<const cd*>(shifts), mode,
                                         reinterpret_cast<cd*>(base), slot,
                                         reinterpret_cast<cd*>(out), ldo, status, nullptr, 0,
                                         h->hnorm2, nullptr, nullptr, nullptr, 0, nullptr, nullptr);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  if (status != nullptr) {
    const int rows = (mode == SSV_G || mode == SSV_TF) ? p : n;
    if (rows > 0) {
      nonfinite_kernel<<<s, 256, 0, st>>>(reinterpret_cast<const cd*>(out), ldo, rows,
                                          m, s, status);
      count_launch();
      SSV_CUDA_TRY(cudaGetLastError());
    }
  }
  return SSV_OK;
}
}  // namespace

size_t noalloc_scratch_bytes() { return kNoAllocScratchBytes; }

int solve_fp64_noalloc(const Handle* h, int s, const double* shifts, const ssv_opts* o,
                       double* out, long long ldo, int* status, cudaStream_t st) {
  const int m = h->m;
  // the same block width as ssv_solve (an autotuned choice included), so the
  // two entry points give the same results
  const int nb = o->nb > 0 ? o->nb : tuned_nb(h->n, m, h->p, SSV_FP64, o->mode);
  if (nb > kNB) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  if (m <= 1) return launch_solve_noalloc<1>(h, s, shifts, nb, o->mode, out, ldo, status, st);
  if (m <= 2) return launch_solve_noalloc<2>(h, s, shifts, nb, o->mode, out, ldo, status, st);
  if (m <= 4) return launch_solve_noalloc<4>(h, s, shifts, nb, o->mode, out, ldo, status, st);
  if (m <= 8) return launch_solve_noalloc<8>(h, s, shifts, nb, o->mode, out, ldo, status, st);
  if (m <= 16) return launch_solve_noalloc<16>(h, s, shifts, nb, o->mode, out, ldo, status, st);
  if (m <= 32) return launch_solve_noalloc<32>(h, s, shifts, nb, o->mode, out, ldo, status, st);
  return SSV_ENOTSUP;
}

}  // namespace ssv

// ---------------------------------------------------------------------------
// Batched solve of many systems (uneven n, m, shift counts) in one persistent
// launch.  A plan fixes the device-side system descriptors, the cost-ordered
// (system, shift) worklist and the scratch, so that running it is one kernel
// launch with fixed arguments (capturable in a CUDA graph and replayable after
// the caller rewrites the shift buffers in place).
// ---------------------------------------------------------------------------
namespace ssv {

struct BatchPlan {
  int dev = 0;
  bool stream_ordered = false;  // buffers from the library pool, ordered on `stream`
  cudaStream_t stream = nullptr;
  int maxm = 1;
  bool dfloat = false;  // SSV_DFLOAT: double-float bulk updates
  int nitems = 0;
  int grid = 0;
  size_t slot = 0;
  size_t smem = 0;
  FpSys* systems = nullptr;
  unsigned long long* items = nullptr;
  cd* scratch = nullptr;
};

namespace {

template <int MAXM, bool DF>
int batch_config(BatchPlan* bp) {
  using L = Layout<MAXM>;
  auto kern = solve_fp64_batch_kernel<MAXM, DF>;
  SSV_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::bytes));
  int per_sm = 0;
  SSV_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L::bytes));
  per_sm = std::max(1, std::min(per_sm, 2));
  bp->grid = std::max(1, std::min(bp->nitems, num_sms() * per_sm));
  bp->smem = L::bytes;
  return SSV_OK;
}

template <int MAXM>
void batch_launch(const BatchPlan* bp, cudaStream_t st) {
  if (bp->dfloat)
    solve_fp64_batch_kernel<MAXM, true><<<bp->grid, kThreads, bp->smem, st>>>(
        bp->systems, bp->items, bp->nitems, bp->scratch, bp->slot);
  else
    solve_fp64_batch_kernel<MAXM, false><<<bp->grid, kThreads, bp->smem, st>>>(
        bp->systems, bp->items, bp->nitems, bp->scratch, bp->slot);
  count_launch();
}

}  // namespace

int batch_create(int nsys, const Handle* const* hs, const int* s, const double* const* shifts,
                 const ssv_opts* o, double* const* outs, const long long* ldos, int* const* status,
                 BatchPlan** out, cudaStream_t stream_ordered) {
  *out = nullptr;
  if ((o->precision != SSV_FP64 && o->precision != SSV_DFLOAT) || o->mode == SSV_X) return SSV_ENOTSUP;
  BatchPlan* bp = new (std::nothrow) BatchPlan();
  if (!bp) return SSV_ENOMEM;
  bp->dfloat = o->precision == SSV_DFLOAT;
  cudaGetDevice(&bp->dev);
  bp->stream_ordered = stream_ordered != nullptr;
  bp->stream = stream_ordered;
  std::vector<FpSys> sys(nsys);
  std::vector<std::pair<double, unsigned long long>> work;
  const bool track_t = (o->mode == SSV_XHAT);
  for (int k = 0; k < nsys; ++k) {
    const Handle* h = hs[k];
    FpSys& d = sys[k];
    d.n = h->n; d.m = h->m; d.p = h->p;
    d.nb = o->nb > 0 ? o->nb : tuned_nb(h->n, h->m, h->p, o->precision, o->mode);
    if (d.nb > kNB || h->m > 32) { delete bp; return SSV_ENOTSUP; }
    d.mode = o->mode; d.H = h->H; d.Ct = h->Ct; d.ldct = h->p > 0 ? h->p : 1; d.R = h->R;
    d.shifts = reinterpret_cast<const cd*>(shifts[k]);
    d.out = reinterpret_cast<cd*>(outs[k]); d.ldo = ldos[k];
    d.status = status ? status[k] : nullptr;
    d.xhat_copy = nullptr; d.ldxc = 0; d.hnorm = h->hnorm2; d.bhat = nullptr; d.ldb = 0;
    d.rhs = nullptr; d.ldr = 0; d.flip_out = 0;
    d.Hhi = h->Hhi; d.Hlo = h->Hlo;
    d.gfull = GivensSched{nullptr, nullptr, 0};
    d.gtail = d.gfull;
    bp->maxm = std::max(bp->maxm, h->m);
    bp->slot = std::max(bp->slot, (size_t)(h->p + h->n) * h->m + (track_t ? (size_t)h->n * h->m : 0));
    const double cost = (double)h->n * h->n * h->m * (1.0 + 2.0 * h->m / d.nb);
    for (int j = 0; j < s[k]; ++j) work.push_back({cost, ((unsigned long long)k << 32) | (unsigned)j});
  }
  std::stable_sort(work.begin(), work.end(),
                   [](const std::pair<double, unsigned long long>& a,
                      const std::pair<double, unsigned long long>& b) { return a.first > b.first; });
  bp->nitems = (int)work.size();
  std::vector<unsigned long long> items(work.size());
  for (size_t i = 0; i < work.size(); ++i) items[i] = work[i].second;
  int rc = SSV_OK;
  const int mm = bp->maxm;
  if (bp->nitems > 0) {
    const bool df = bp->dfloat;
    if (mm <= 1) rc = df ? batch_config<1, true>(bp) : batch_config<1, false>(bp);
    else if (mm <= 2) rc = df ? batch_config<2, true>(bp) : batch_config<2, false>(bp);
    else if (mm <= 4) rc = df ? batch_config<4, true>(bp) : batch_config<4, false>(bp);
    else if (mm <= 8) rc = df ? batch_config<8, true>(bp) : batch_config<8, false>(bp);
    else if (mm <= 16) rc = df ? batch_config<16, true>(bp) : batch_config<16, false>(bp);
    else rc = df ? batch_config<32, true>(bp) : batch_config<32, false>(bp);
  }
  cudaError_t e = cudaSuccess;
  if (rc == SSV_OK && bp->nitems > 0) {
    if (bp->stream_ordered) {
      // stream-ordered: no device-wide synchronisation, so concurrent batches on
      // other streams keep running; pageable sources are consumed before return
      cudaStream_t st = bp->stream;
      e = pool_alloc((void**)&bp->systems, sizeof(FpSys) * nsys, st);
      if (e == cudaSuccess)
        e = pool_alloc((void**)&bp->items, sizeof(unsigned long long) * items.size(), st);
      if (e == cudaSuccess)
        e = pool_alloc((void**)&bp->scratch, sizeof(cd) * bp->slot * bp->grid, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(bp->systems, sys.data(), sizeof(FpSys) * nsys, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(bp->items, items.data(), sizeof(unsigned long long) * items.size(),
                            cudaMemcpyHostToDevice, st);
    } else {
      e = cudaMalloc((void**)&bp->systems, sizeof(FpSys) * nsys);
      if (e == cudaSuccess) e = cudaMalloc((void**)&bp->items, sizeof(unsigned long long) * items.size());
      if (e == cudaSuccess) e = cudaMalloc((void**)&bp->scratch, sizeof(cd) * bp->slot * bp->grid);
      if (e == cudaSuccess)
        e = cudaMemcpy(bp->systems, sys.data(), sizeof(FpSys) * nsys, cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(bp->items, items.data(), sizeof(unsigned long long) * items.size(),
                       cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
      set_cuda_error(e);
      rc = e == cudaErrorMemoryAllocation ? SSV_ENOMEM : SSV_ECUDA;
    }
  }
  if (rc != SSV_OK) {
    batch_destroy(bp);
    return rc;
  }
  *out = bp;
  return SSV_OK;
}

int batch_run(const BatchPlan* bp, cudaStream_t st) {
  if (bp->nitems == 0) return SSV_OK;
  const int mm = bp->maxm;
  if (mm <= 1) batch_launch<1>(bp, st);
  else if (mm <= 2) batch_launch<2>(bp, st);
  else if (mm <= 4) batch_launch<4>(bp, st);
  else if (mm <= 8) batch_launch<8>(bp, st);
  else if (mm <= 16) batch_launch<16>(bp, st);
  else batch_launch<32>(bp, st);
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

void batch_destroy(BatchPlan* bp) {
  if (!bp) return;
  if (bp->stream_ordered) {
    if (bp->systems) cudaFreeAsync(bp->systems, bp->stream);
    if (bp->items) cudaFreeAsync(bp->items, bp->stream);
    if (bp->scratch) cudaFreeAsync(bp->scratch, bp->stream);
  } else {
    cudaFree(bp->systems);
    cudaFree(bp->items);
    cudaFree(bp->scratch);
  }
  delete bp;
}

// ---------------------------------------------------------------------------
// Autotuner for the elimination block width n_b: times each candidate on the
// caller's shifts with CUDA events and caches the fastest per
// (n, m, p, precision, mode) for the life of the process.
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
  int n, m, p, prec, mode;
  bool operator<(const TuneKey& o) const {
    if (n != o.n) return n < o.n;
    if (m != o.m) return m < o.m;
    if (p != o.p) return p < o.p;
    if (prec != o.prec) return prec < o.prec;
    return mode < o.mode;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
}  // namespace

int tuned_nb(int n, int m, int p, int prec, int mode) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(TuneKey{n, m, p, prec, mode});
  return it == g_tune.end() ? default_nb(n, m) : it->second;
}

int autotune_nb(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                long long ldo, cudaStream_t st, int* best_nb, float* best_ms) {
  static const int cand_fp64[] = {32, 48, 64, 96, 128};
  static const int cand_mixed[] = {16, 24, 32, 48, 64};
  const int* cand = o->precision == SSV_MIXED ? cand_mixed : cand_fp64;
  cudaEvent_t e0, e1;
  SSV_CUDA_TRY(cudaEventCreate(&e0));
  SSV_CUDA_TRY(cudaEventCreate(&e1));
  int best = default_nb(h->n, h->m);
  float bms = 1e30f;
  int rc = SSV_OK;
  for (int ci = 0; ci < 5; ++ci) {
    const int c = cand[ci];
    ssv_opts oo = *o;
    oo.nb = c;
    for (int rep = 0; rep < 2 && rc == SSV_OK; ++rep) {  // first run warms up
      cudaEventRecord(e0, st);
      rc = oo.precision == SSV_MIXED ? solve_mixed(h, s, shifts, &oo, out, ldo, nullptr, nullptr, st)
                                     : solve_fp64(h, s, shifts, &oo, out, ldo, nullptr, nullptr, st);
      cudaEventRecord(e1, st);
      if (rc == SSV_OK && cudaEventSynchronize(e1) == cudaSuccess && rep == 1) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < bms) { bms = ms; best = c; }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SSV_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[TuneKey{h->n, h->m, h->p, o->precision, o->mode}] = best;
  }
  *best_nb = best;
  if (best_ms) *best_ms = bms;
  return SSV_OK;
}

}  // namespace ssv
