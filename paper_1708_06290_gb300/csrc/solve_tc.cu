// Shift-batched sweep with the trailing update on the tensor cores.
//
// The sweep of Sec. 3.1 / Algorithm 8 for every shift, run as the paper runs
// it on a GPU: one phase per block step k for all shifts at once, so that the
// update of the rows above the block ("Step 2, revisited": one GEMM with the
// shared operand Z1 = [Ct; H](1:r, fresh columns) and every shift's block
// transform, Z2 <- Z1 P1 + Z2 P2 - sigma E P1) multiplies a tile of H that is
// staged once for a group of shifts.  Per block step:
//
//   1. panel (one thread block per shift, three per SM): the n_b x (n_b + m) window block is
//      triangularised bottom-up by one complex Householder reflector per row
//      over the m + 1 candidate columns (double-word reflector scalars,
//      double-float application, as in the double-float sweep), giving the
//      coefficients P1 (n_b x m) and P2 (m x m).  The panel also updates the p
//      rows of Ct (small), writes P1 as BF16 digit tiles, and keeps the P1
//      rows and P2 that the X-hat back pass needs;
//   2. update (persistent, one thread block per SM): work items of 128 rows
//      of H x one group of shifts (N = 64 real columns: each shift's m complex
//      columns as 2m real ones, padded to a power of two).  Z1 P1 is formed
//      exactly as in the tensor-core residual (error-free splitting after
//      Ozaki, Ogita, Oishi and Rump): H's rows and P1's real columns are
//      written as 7-bit digits relative to a power-of-two scale (eight for a
//      row of H, seven for a column of P1), each digit exact in BF16, and the
//      35 digit products H_k P_l with k + l <= 7 run as tcgen05.mma (BF16 x
//      BF16 -> FP32, M = 128, N = 64, K = 16) into eight TMEM accumulators, one
//      per level k + l, where every partial sum is an integer below
//      7 * 128 * 127^2 < 2^24 and therefore exact.  The
//      digit tiles reach shared memory by 1-D TMA bulk copies on an mbarrier,
//      two stages in flight.  The epilogue reads the levels back (tcgen05.ld),
//      adds them scaled by 2^{-7 t} into double-float sums, scales by the row
//      and column exponents, and adds Z2 P2 and the shifted-diagonal
//      correction in double-float on the FP32 pipe;
//   3. after the last block: the final m x m block, G = Ct Xhat or X-hat by the
//      backward pass over the stored block transforms.
//
// Accuracy: the digits beyond the eighth of H and the seventh of P1 and the
// products of level > 7 are dropped, about 2^-49 of the row scale times the
// column scale (the double-float class of the SSV_DFLOAT sweep).  H's rows get
// all eight digits because a dominant diagonal sets the row scale: the
// off-diagonal entries of a row can be 2^7 below it.  The first block holds
// (n - m) mod n_b rows (n_b when that is 0), so that every later block starts
// at a column that is a multiple of n_b and the H digit tiles (32 columns
// deep) line up with the fresh columns.
#include <algorithm>

#include "dfloat.cuh"
#include "ssv_internal.cuh"
#include "tc_common.cuh"

namespace ssv {

namespace {

using namespace tcg;

// Debug builds (-DSSV_BOUNDS_CHECK): every global index of the sweep's kernels
// is checked against its buffer; an index out of range sets bit 1 of the
// solve's error word (every shift of the solve then reports a non-finite
// result) and is replaced by 0, so the access stays inside the buffer.  In
// normal builds BCK(i, n) is i.
#ifdef SSV_BOUNDS_CHECK
__device__ __forceinline__ size_t bck(long long i, size_t n, int* err) {
  if (i < 0 || (size_t)i >= n) {
    atomicOr(err, 2);
    return 0;
  }
  return (size_t)i;
}
#define BCK(i, n) bck((long long)(i), (size_t)(n), a.err)
#else
#define BCK(i, n) ((size_t)(i))
#endif

constexpr int kPT = 256;             // threads of the setup, panel and final kernels
constexpr int kNBT = 128;            // n_b of the tensor-core sweep (K of the update)
constexpr int kMaxM = kTcMaxM;       // m <= 16
constexpr int kSlots = kMaxM + 1;    // m live + the fresh column
constexpr int kCoefRows = kNBT + kMaxM;
constexpr int kUM = 128;             // H rows per update item = TMEM lanes
// real columns per update item (shift group): 64 = one update block per SM with
// two stage buffers; 32 = two blocks per SM with one stage buffer each, so that
// one block's epilogue runs under the other's products
#ifndef SSV_TCS_N
#define SSV_TCS_N 64
#endif
constexpr int kUN = SSV_TCS_N;
static_assert(kUN == 32 || kUN == 64, "update item width");
constexpr int kBufU = kUN == 64 ? 2 : 1;   // stage buffers of an update block
constexpr int kCtasU = kUN == 64 ? 1 : 2;  // update blocks per SM
constexpr int kKS = 32;              // K per shared-memory stage
constexpr int kKG = kKS / 8;         // core matrices along K in a tile
constexpr int kSDH = 8;              // digits of H (all eight slices of its digit tiles)
constexpr int kSD = 7;               // digits of the block transforms' columns
constexpr int kLev = 8;              // levels k + l = 0 .. 7
constexpr int kStages = kNBT / kKS;  // stages per block step
constexpr int kAT = kUM * kKS;       // BF16 elements of one H digit tile
constexpr int kBT = kUN * kKS;       // BF16 elements of one P1 digit tile
#ifndef SSV_TCS_FUSED
#define SSV_TCS_FUSED 1  // 1: Z1 P1 as fused-level products (one per H digit and <= 256 columns)
#endif
// a stage: eight H digit tiles, seven P1 digit tiles and (fused form) one tile of
// zeros standing for P1 digit 7, so that the H digit 0 products reach all levels
constexpr int kBPlanes = SSV_TCS_FUSED ? kSD + 1 : kSD;
constexpr uint32_t kStageBytes = (uint32_t)(kSDH * kAT + kBPlanes * kBT) * 2;
constexpr uint32_t kLoadBytes = (uint32_t)(kSDH * kAT + kSD * kBT) * 2;  // copied per stage
constexpr uint32_t kZeroOff = kLoadBytes;                                 // the zero tile in a stage
constexpr int kIss = 4;              // threads issuing products (lane 0 of warps 0..3)
constexpr uint32_t kIdescU = idesc_bf16(kUM, kUN);
constexpr int kTmemCols = 8 * kUN;   // 8 levels x kUN columns
// polls of one mbarrier wait before the update gives up (a stage's copies and
// products complete within microseconds)
constexpr long long kUpdWait = 1LL << 22;
static_assert(kLev * kUN <= kTmemCols, "TMEM columns of the levels");
// dynamic shared memory of the update, in this order: two stage buffers (later
// the group's Z2 and P2 digit tiles); the group's P2 / sigma rows (S * 2 m^2 <=
// 64 m float4); the column exponents of P1 and of P2's real form (kUN ints
// each); the row maxima of the quarters (4 x 128 floats); the shifts (at most
// kUN); kIss + 3 mbarriers; the TMEM address slot
constexpr size_t kOffPc = (size_t)kBufU * kStageBytes;
constexpr size_t kPcF4 = (size_t)kUN * kMaxM;
constexpr size_t kOffExp = kOffPc + kPcF4 * 16;
constexpr size_t kOffExp2 = kOffExp + (size_t)kUN * sizeof(int);
constexpr size_t kOffXmax = kOffExp2 + (size_t)kUN * sizeof(int);
constexpr size_t kOffSig = kOffXmax + (size_t)4 * kUM * sizeof(float);
constexpr size_t kOffBar = kOffSig + (size_t)kUN * 16;
constexpr size_t kOffSlot = kOffBar + (size_t)(kIss + 3) * 8;
constexpr size_t kUpdSmem = kOffSlot + 16;
static_assert(kOffBar % 8 == 0 && kOffSig % 16 == 0, "alignment of the smem carve-up");
static_assert(kCtasU * (kUpdSmem + 1024) <= 228 * 1024, "shared memory of the update blocks");
// the Z2 / P2 digit tiles of a group (S shifts, 7 digits, 128 x cs and cs x cs) reuse the stage buffers
static_assert(7 * (128 * 32 + 32 * 32) * 2 * (kUN / 32) <= kBufU * (size_t)kStageBytes, "Z2 P2 tiles");
static_assert(7 * (128 * 16 + 16 * 16) * 2 * (kUN / 16) <= kBufU * (size_t)kStageBytes, "Z2 P2 tiles");

// element offset in a K-major core-matrix tile (8 rows x 8 K per 128 bytes;
// byte strides 128 along K, kKG * 128 along rows): the layout of the residual's
// H digit tiles
__host__ __device__ __forceinline__ int tile_off(int row, int k) {
  return (((row >> 3) * kKG + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7);
}

// products of level t: H digit k, transform digit t - k, k in [max(0, t - 6), min(7, t)]
// (1, 2, 3, 4, 5, 6, 7, 7 for t = 0 .. 7); issuer owning level t:
// {7, 1}, {6, 0}, {5, 2}, {4, 3} (9, 8, 9, 9 products)
__host__ __device__ constexpr int level_owner(int t) {
  return (t == 7 || t == 1) ? 0 : (t == 6 || t == 0) ? 1 : (t == 5 || t == 2) ? 2 : 3;
}

// column stride of one shift in a group: 2m real columns rounded up to a power of two
__host__ __device__ inline int shift_cols(int m) {
  int c = 2;
  while (c < 2 * m) c <<= 1;
  return c;
}

struct TcsArgs {
  int n, m, p, s, cs, S, ngroups, mode;
  const double* H;       // n x n
  const float* Hhi;      // double-float split of H
  const float* Hlo;
  const double* Ct;      // p x n (ld ldct)
  int ldct;
  const double* R;       // n x m
  const cd* shifts;
  const double* hnorm;   // ||H||_F^2, trace(H)
  float4* Z2;            // per shift: (p + n) x m double-float window columns, ld p + n
  cd* ZT;                // per shift: n x m rows P1 of every step (X-hat mode), or null
  size_t z2_stride;      // float4 per shift slot
  uint16_t* Pd;          // P1 digit tiles: [group][digit][stage][kBT]
  int* pexp;             // per shift: 2m column exponents (stride 2 kMaxM)
  float4* pc;            // per shift: P2 (m x m) then sigma rows P1(0:min(m,nbe), :) (m x m)
  cd* out;
  long long ldo;
  int* flags;            // per shift: 1 = singular to working precision
  int* status;
  const uint4* Hs;       // H digit tiles (residual layout) and row exponents
  const int* hexp;
  int RB, KT;            // row blocks / K blocks of the H digit tiles
  int* err;              // an update wait gave up
  // Z2 P2 on the tensor cores (cs >= 16, m >= 5): the H rows of every shift's
  // window columns as digit tiles (row-scaled, K = cs real entries interleaved
  // Re, Im) and the real form of each step's P2 (column-scaled, cs x cs)
  int tcz;
  int npad;
  uint16_t* Zd;          // [shift][row block][digit][128 x cs]
  int* zexp;             // [shift][npad] row exponents
  uint16_t* P2d;         // [shift][digit][cs x cs]
  int* p2exp;            // [shift][2 kMaxM] column exponents
  // buffer sizes (elements) for the debug build's index checks
  size_t n_z2, n_zt, n_pd, n_zd, n_p2d, n_pc, n_hs, n_out;
};

// digit tiles of window row p + i (H row i) of shift sh, from the double-float
// values Z2f(p + i, q): the row exponent over the 2m real entries, seven
// digits of each entry at K = 2q (Re), 2q + 1 (Im), zero up to cs
__device__ void write_z2_digits(const TcsArgs& a, int sh, int i, const float4* Z2f, int ldz) {
  const int m = a.m, cs = a.cs, kg = cs / 8;
  float mx = 0.f;
  for (int q = 0; q < m; ++q) {
    const float4 z = Z2f[BCK((a.p + i) + (size_t)q * ldz, a.z2_stride)];
    mx = fmaxf(mx, fmaxf(fabsf(z.x), fabsf(z.z)));
    if (!(fabsf(z.x) <= 3.4e38f) || !(fabsf(z.z) <= 3.4e38f)) mx = __int_as_float(0x7f800000);
  }
  const int E = scale_exp_f(mx);
  a.zexp[BCK((size_t)sh * a.npad + i, (size_t)a.s * a.npad)] = E;
  const size_t T0 = ((size_t)sh * a.RB + i / 128) * 7 * (128 * cs);
  for (int k8 = 0; k8 < cs; k8 += 8) {
    unsigned short dg[8][7];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int kk = k8 + e, q = kk >> 1;
      float hi = 0.f, lo = 0.f;
      if (q < m) {
        const float4 z = Z2f[BCK((a.p + i) + (size_t)q * ldz, a.z2_stride)];
        hi = (kk & 1) ? z.z : z.x;
        lo = (kk & 1) ? z.w : z.y;
      }
      digits7_pair(hi, lo, E, dg[e]);
    }
    const int off = tile_off_kg(i % 128, k8, kg);
#pragma unroll
    for (int l = 0; l < 7; ++l) {
      uint4 u;
      u.x = dg[0][l] | ((unsigned)dg[1][l] << 16);
      u.y = dg[2][l] | ((unsigned)dg[3][l] << 16);
      u.z = dg[4][l] | ((unsigned)dg[5][l] << 16);
      u.w = dg[6][l] | ((unsigned)dg[7][l] << 16);
      *reinterpret_cast<uint4*>(a.Zd + BCK(T0 + (size_t)l * (128 * cs) + off, a.n_zd)) = u;
    }
  }
}

__device__ __forceinline__ double shifted_norm2(const double* hnorm, int n, cd sg) {
  return fmax(hnorm[0] - 2.0 * sg.x * hnorm[1] + (double)n * (sg.x * sg.x + sg.y * sg.y), 0.0);
}

// ---- setup: Z2 = last m columns of [Ct; H] - sigma on the diagonal ---------
__global__ void __launch_bounds__(kPT) tcs_setup_kernel(TcsArgs a) {
  const int sh = blockIdx.x;
  const int n = a.n, m = a.m, p = a.p, ldz = p + n;
  const cd sigma = a.shifts[sh];
  float4* Z2 = a.Z2 + (size_t)sh * a.z2_stride;
  for (long long idx = threadIdx.x; idx < (long long)ldz * m; idx += kPT) {
    const int i = (int)(idx % ldz), q = (int)(idx / ldz);
    const int j = n - m + q;
    const double v = i < p ? a.Ct[i + (size_t)j * a.ldct] : a.H[(i - p) + (size_t)j * n];
    cd z = mkcd(v, 0.0);
    if (i - p == j) z = csub(z, sigma);
    Z2[BCK(idx, a.z2_stride)] = df_split(z);
  }
  if (threadIdx.x == 0) a.flags[sh] = 0;
  if (a.tcz) {
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += kPT) write_z2_digits(a, sh, i, Z2, ldz);
  }
}

// ---- panel of block step `step` (1-based), rows k - nbe .. k - 1 ------------
struct PanelSmem {
  float4 cand[kSlots * kNBT];
  float4 coef[kCoefRows * kSlots];
  float4 vf[kMaxM + 4];
  int fexp[2 * kMaxM];
  int f2exp[2 * kMaxM];
  int sing;
};

__global__ void __launch_bounds__(kPT, 3) tcs_panel_kernel(TcsArgs a, int k, int nbe, int step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PanelSmem& sm = *reinterpret_cast<PanelSmem*>(smem_raw);
  constexpr int S = kSlots;
  const int sh = blockIdx.x;
  const int tid = threadIdx.x;
  const int n = a.n, m = a.m, p = a.p, ldz = p + n;
  const int r = p + k - nbe;       // rows of [Ct; M] above the block
  const int j0 = k - m - nbe;      // first fresh column
  const cd sigma = a.shifts[sh];
  float4* Z2f = a.Z2 + (size_t)sh * a.z2_stride;
  const double sing_tol = (double)n * 7.105427357601002e-15 * sqrt(shifted_norm2(a.hnorm, n, sigma));
  const float sing_tol_f = (float)sing_tol;
  const float* __restrict__ Hhi = a.Hhi;
  const float* __restrict__ Hlo = a.Hlo;
  auto split4 = [](cd z) -> float4 { return df_split(z); };
  // entry (global row gr, fresh column jc) of H - sigma I as FP32 pairs
  auto fresh4 = [&](int gr, int jc) -> float4 {
    const size_t hidx = (size_t)gr + (size_t)jc * n;
    if (gr == jc) return split4(csub(mkcd((double)Hhi[hidx] + (double)Hlo[hidx], 0.0), sigma));
    return make_float4(Hhi[hidx], Hlo[hidx], 0.f, 0.f);
  };
  float4* cand4 = sm.cand;
  float4* coef4 = sm.coef;
  float4* vf = sm.vf;
  if (tid == 0) sm.sing = 0;
  for (int idx = tid; idx < m * nbe; idx += kPT) {
    const int t = idx % nbe, q = idx / nbe;
    cand4[q * kNBT + t] = Z2f[BCK((r + t) + (size_t)q * ldz, a.z2_stride)];
  }
  for (int idx = tid; idx < kCoefRows * S; idx += kPT) {
    const int c = idx / S, slot = idx % S;
    const bool one = (slot < m && c == kNBT + slot) || (slot == m && c == nbe - 1);
    coef4[idx] = make_float4(one ? 1.f : 0.f, 0.f, 0.f, 0.f);
  }
  {
    const int c = nbe - 1, jc = j0 + c;
    for (int t = tid; t <= c; t += kPT) cand4[m * kNBT + t] = fresh4(k - nbe + t, jc);
  }
  __syncthreads();
  for (int c = nbe - 1; c >= 0; --c) {
    const int fs = m;                         // slot of the fresh column of row c
    // the next fresh column is read now, its latency hidden behind this row
    float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c > 0 && tid < c) pre = fresh4(k - nbe + tid, j0 + c - 1);
    if (tid < 32) {
      // reflector scalars in double-word arithmetic:
      //   v = conj(x) + e^{i arg conj(x_f)} ||x|| e_f,  tau = 1 / (||x||^2 + |x_f| ||x||)
      dw rest2{0.f, 0.f};
      for (int q = tid; q < m; q += 32) {
        const float4 x = cand4[q * kNBT + c];
        df_mac(rest2.hi, rest2.lo, x.x, x.y, x.x, x.y);
        df_mac(rest2.hi, rest2.lo, x.z, x.w, x.z, x.w);
        vf[q] = make_float4(x.x, x.y, -x.z, -x.w);
      }
      rest2 = dw_fast(rest2.hi, rest2.lo);
      for (int o = 16; o > 0; o >>= 1)
        rest2 = dw_add(rest2, dw{__shfl_xor_sync(0xffffffffu, rest2.hi, o),
                                 __shfl_xor_sync(0xffffffffu, rest2.lo, o)});
      if (tid == 0) {
        const float4 xf = cand4[fs * kNBT + c];
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
        vf[kMaxM + 2] = make_float4(tau.hi, tau.lo, 0.f, 0.f);
        if (nrm.hi <= sing_tol_f) sm.sing = 1;
      }
    }
    __syncthreads();
    const float4 tauf = vf[kMaxM + 2];
    {
      const int nrow = c;
      const int ncoef = (nbe - c) + m;
      // nrow + ncoef <= n_b + m < kPT: each thread has at most one row e = tid,
      // and the thread of window row e < c holds that row's next fresh entry
      for (int e = tid; e < nrow + ncoef; e += kPT) {
        float4* base;
        int stride;
        if (e < nrow) {
          base = cand4 + e;
          stride = kNBT;
        } else {
          const int ee = e - nrow;
          const int crow = ee < nbe - c ? c + ee : kNBT + (ee - (nbe - c));
          base = coef4 + crow * S;
          stride = 1;
        }
        if (tauf.x != 0.0f) {
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
          const float sr = xrh + xrl, si = xih + xil;
          x = make_float4(sr, xrl - (sr - xrh), si, xil - (si - xih));
          base[slot * stride] = x;
        }
        }
        // the eliminated column is done with: its slot takes the next fresh
        // column, whose coefficients are e_{c-1} (row c - 1 is set below; the
        // rows this loop covers get zero, every other row is zero already)
        base[fs * stride] = e < nrow ? pre : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (c > 0 && tid == 0) coef4[(c - 1) * S + fs] = make_float4(1.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
  }
  // coef rows c < nbe hold P1(c, :), rows kNBT + qq hold P2(qq, :) (slots 0..m-1)

  // ---- P1 as BF16 digit tiles: column exponents first (one warp per real column)
  const int warp = tid >> 5, lane = tid & 31;
  for (int cr = warp; cr < 2 * m; cr += kPT / 32) {
    const int q = cr >> 1;
    double mx = 0.0;
    bool bad = false;
    for (int c = lane; c < nbe; c += 32) {
      const float4 w = coef4[c * S + q];
      const double v = fabs((cr & 1) ? (double)w.z + (double)w.w : (double)w.x + (double)w.y);
      if (!(v <= 1.7976931348623157e308)) bad = true;
      else mx = fmax(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bad = __shfl_xor_sync(0xffffffffu, (int)bad, o) || bad;
    }
    if (lane == 0) {
      const int E = bad ? kBadExp : scale_exp(mx);
      sm.fexp[cr] = E;
      a.pexp[BCK((size_t)sh * 2 * kMaxM + cr, (size_t)a.s * 2 * kMaxM)] = E;
    }
  }
  __syncthreads();
  {
    // item = (real column cr, 8 consecutive K rows): seven uint4 stores
    const int g = sh / a.S, slot_row = (sh % a.S) * a.cs;
    const size_t Pg0 = (size_t)g * kSD * kStages * kBT;
    for (int it = tid; it < 2 * m * (kNBT / 8); it += kPT) {
      const int cr = it / (kNBT / 8), c8 = (it % (kNBT / 8)) * 8;
      const int q = cr >> 1, E = sm.fexp[cr];
      unsigned short dg[8][kDigits];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int c = c8 + e;
        double v = 0.0;
        if (c < nbe) {
          const float4 w = coef4[c * S + q];
          v = (cr & 1) ? (double)w.z + (double)w.w : (double)w.x + (double)w.y;
        }
        digits8(v, E, dg[e]);
      }
      const int J = c8 / kKS;
      const int off = tile_off(slot_row + cr, c8 % kKS);
#pragma unroll
      for (int l = 0; l < kSD; ++l) {
        uint4 u;
        u.x = dg[0][l] | ((unsigned)dg[1][l] << 16);
        u.y = dg[2][l] | ((unsigned)dg[3][l] << 16);
        u.z = dg[4][l] | ((unsigned)dg[5][l] << 16);
        u.w = dg[6][l] | ((unsigned)dg[7][l] << 16);
        *reinterpret_cast<uint4*>(a.Pd + BCK(Pg0 + ((size_t)l * kStages + J) * kBT + off, a.n_pd)) = u;
      }
    }
  }
  // ---- P2 and the sigma rows for the update's epilogue
  {
    float4* pc = a.pc + (size_t)sh * 2 * kMaxM * kMaxM;
    const int nsig = min(m, nbe);
    for (int e = tid; e < 2 * m * m; e += kPT) {
      const int row = e / m, q = e % m;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < m) v = coef4[(kNBT + row) * S + q];
      else if (row - m < nsig) v = coef4[(row - m) * S + q];
      pc[e] = v;
    }
  }
  // ---- Z2 P2 on the tensor cores: P2's real form (cs x cs, entry (K = 2qq + ri,
  //      N = 2q + ro) from P2(qq, q): Re for ri = ro, -Im for (1, 0), Im for
  //      (0, 1)) as seven-digit tiles, column-scaled
  if (a.tcz) {
    const int cs = a.cs, kg = cs / 8;
    for (int c = tid; c < cs; c += kPT) {
      const int q = c >> 1;
      float mx = 0.f;
      if (q < m) {
        for (int qq = 0; qq < m; ++qq) {
          const float4 w = coef4[(kNBT + qq) * S + q];
          mx = fmaxf(mx, fmaxf(fabsf(w.x), fabsf(w.z)));
          if (!(fabsf(w.x) <= 3.4e38f) || !(fabsf(w.z) <= 3.4e38f)) mx = __int_as_float(0x7f800000);
        }
      }
      const int E = scale_exp_f(mx);
      sm.f2exp[c] = E;
      a.p2exp[BCK((size_t)sh * 2 * kMaxM + c, (size_t)a.s * 2 * kMaxM)] = E;
    }
    __syncthreads();
    const size_t T0 = (size_t)sh * 7 * cs * cs;
    for (int it = tid; it < cs * (cs / 8); it += kPT) {
      const int c = it / (cs / 8), k8 = (it % (cs / 8)) * 8;
      const int q = c >> 1, ro = c & 1, E = sm.f2exp[c];
      unsigned short dg[8][7];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int kk = k8 + e, qq = kk >> 1, ri = kk & 1;
        float hi = 0.f, lo = 0.f;
        if (q < m && qq < m) {
          const float4 w = coef4[(kNBT + qq) * S + q];
          if (ri == ro) { hi = w.x; lo = w.y; }
          else if (ri == 1) { hi = -w.z; lo = -w.w; }
          else { hi = w.z; lo = w.w; }
        }
        digits7_pair(hi, lo, E, dg[e]);
      }
      const int off = tile_off_kg(c, k8, kg);
#pragma unroll
      for (int l = 0; l < 7; ++l) {
        uint4 u;
        u.x = dg[0][l] | ((unsigned)dg[1][l] << 16);
        u.y = dg[2][l] | ((unsigned)dg[3][l] << 16);
        u.z = dg[4][l] | ((unsigned)dg[5][l] << 16);
        u.w = dg[6][l] | ((unsigned)dg[7][l] << 16);
        *reinterpret_cast<uint4*>(a.P2d + BCK(T0 + (size_t)l * cs * cs + off, a.n_p2d)) = u;
      }
    }
  }
  // ---- X-hat mode: P1 rows into ZT, P2 parked in this shift's output rows
  //      n - step m .. n - (step - 1) m - 1 (read back before the back pass
  //      writes them, since every later block is at least m rows high)
  if (a.mode == SSV_XHAT) {
    cd* ZT = a.ZT + (size_t)sh * (size_t)n * m;
    for (int idx = tid; idx < nbe * m; idx += kPT) {
      const int c = idx % nbe, q = idx / nbe;
      ZT[BCK((j0 + c) + (size_t)q * n, (size_t)n * m)] = df_join(coef4[c * S + q]);
    }
    cd* tout = a.out + (size_t)sh * m * a.ldo;
    for (int idx = tid; idx < m * m; idx += kPT) {
      const int qq = idx % m, q = idx / m;
      tout[BCK(n - step * m + qq, n) + (size_t)q * a.ldo] = df_join(coef4[(kNBT + qq) * S + q]);
    }
  }
  // ---- the p rows of Ct: Z2(i, :) = Ct(i, fresh) P1 + Z2(i, :) P2, double-float,
  //      in chunks of whole rows (each entry reads its row's old values)
  const int rows_per_chunk = max(1, (2 * kPT) / m);
  for (int i0 = 0; i0 < p; i0 += rows_per_chunk) {
  const int ic = min(rows_per_chunk, p - i0);
  float4 nv[2];
  int nitem = 0;
  for (int e = tid; e < ic * m && nitem < 2; e += kPT, ++nitem) {
    const int i = i0 + e / m, q = e % m;
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    for (int c = 0; c < nbe; ++c) {
      const double z = a.Ct[i + (size_t)(j0 + c) * a.ldct];
      const float zh = (float)z, zl = (float)(z - (double)zh);
      const float4 w = coef4[c * S + q];
      df_mac(rh, rl, zh, zl, w.x, w.y);
      df_mac(ih, il, zh, zl, w.z, w.w);
    }
    for (int qq = 0; qq < m; ++qq) {
      const float4 zz = Z2f[BCK(i + (size_t)qq * ldz, a.z2_stride)];
      const float4 w = coef4[(kNBT + qq) * S + q];
      df_mac(rh, rl, zz.x, zz.y, w.x, w.y);
      df_mac(rh, rl, -zz.z, -zz.w, w.z, w.w);
      df_mac(ih, il, zz.x, zz.y, w.z, w.w);
      df_mac(ih, il, zz.z, zz.w, w.x, w.y);
    }
    const float sr = rh + rl, si = ih + il;
    nv[nitem] = make_float4(sr, rl - (sr - rh), si, il - (si - ih));
  }
  __syncthreads();  // every old entry of these rows is read before any is written
  nitem = 0;
  for (int e = tid; e < ic * m && nitem < 2; e += kPT, ++nitem) {
    const int i = i0 + e / m, q = e % m;
    Z2f[BCK(i + (size_t)q * ldz, a.z2_stride)] = nv[nitem];
  }
  __syncthreads();
  }
  if (tid == 0 && sm.sing) a.flags[sh] = 1;
}

// ---- update of the H rows above the block: Z2 <- Z1 P1 + Z2 P2 - sigma E P1 --
// the level sums of one thread's 16 TMEM columns (lane = its row), each level t
// scaled by 2^{-7 (t + 2)} and added into double-float sums
static __device__ __forceinline__ void drain_levels(uint32_t tl, int nlev, float (&ah)[16],
                                                    float (&al)[16], int lstride = kUN) {
#pragma unroll
  for (int c = 0; c < 16; ++c) { ah[c] = 0.f; al[c] = 0.f; }
  float sc = 0.0078125f * 0.0078125f;  // 2^{-7 (t + 2)}, t = 0
#pragma unroll 1
  for (int lv = 0; lv < nlev; ++lv) {
    uint32_t rr[16];
    tmem_ld16(tl + (uint32_t)(lv * lstride), rr);
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float pv = __uint_as_float(rr[c]) * sc;
      const float s2 = ah[c] + pv;
      const float bp = s2 - ah[c];
      al[c] += (ah[c] - (s2 - bp)) + (pv - bp);
      ah[c] = s2;
    }
    sc *= 0.0078125f;
  }
}

constexpr int kUT = (kUN / 16) * kUM;  // update threads: one per H row of the tile and 16 columns

// The update of block step (k, nbe).  TCZ: Z2 P2 as a second round of digit
// products on the tensor cores (m >= 5); otherwise in double-float in the
// epilogue.  Per item (row tile I, group g):
//   1. the stages of Z1 P1 (H digit tiles x P1 digit tiles) into the eight
//      TMEM levels, two stage buffers in flight;
//   2. TCZ: the group's Z2 and P2 digit tiles are copied into the (then free)
//      stage buffers while the threads drain the Z1 P1 levels into
//      double-float sums; then the 28 products of Z2 P2 per shift go into
//      seven TMEM levels, are drained and added;
//   3. the next item's first stage streams in during the rest of the epilogue:
//      the shifted-diagonal correction, the new Z2 rows in double-float and
//      (TCZ) as digit tiles for the next block step.
template <bool TCZ>
__global__ void __launch_bounds__(kUT, kCtasU) tcs_update_kernel(TcsArgs a, int k, int nbe) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int n = a.n, m = a.m, p = a.p, ldz = p + n;
  const int hrows = k - nbe;              // H rows above the block
  const int j0 = k - m - nbe;             // first fresh column (a multiple of 32)
  const int nsig = min(m, nbe);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int S = a.S, cs = a.cs, G = a.ngroups;
  // an earlier launch of this solve gave up a wait: its results are void, skip
  // (the flag is read by every thread and combined, so the whole block agrees)
  if (__syncthreads_or(*(volatile int*)a.err != 0)) return;
  const int RT = (hrows + kUM - 1) / kUM;
  const long long items = (long long)RT * G;
  const int nst = (nbe + kKS - 1) / kKS;
  const int JH0 = j0 / kKS;
  float4* pcs = reinterpret_cast<float4*>(smem + kOffPc);                   // S x 2 m m
  int* fexp = reinterpret_cast<int*>(smem + kOffExp);                        // kUN
  int* f2exp = reinterpret_cast<int*>(smem + kOffExp2);                      // kUN
  float* xmax = reinterpret_cast<float*>(smem + kOffXmax);                   // 4 x 128
  cd* sig = reinterpret_cast<cd*>(smem + kOffSig);                           // <= kUN shifts
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + kOffBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kOffSlot);
  const uint32_t mb = smem_addr(mbar);        // kIss MMA barriers, two stage loads, one Z2 / P2 load
  const uint32_t lmb0 = mb + 8u * kIss;
  const uint32_t lmb2 = mb + 8u * (kIss + 2);
  const uint32_t sBase = smem_addr(smem);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kIss + 3; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb + 8u * q));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // the zero tiles of the stage buffers (fused form; the copies never write them)
  auto zero_tile = [&](int b) {
    if (!SSV_TCS_FUSED) return;
    uint4* zp = reinterpret_cast<uint4*>(smem + (size_t)b * kStageBytes + kZeroOff);
    for (int e = tid; e < kBT * 2 / 16; e += kUT) zp[e] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  };
  for (int b = 0; b < kBufU; ++b) zero_tile(b);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  uint32_t mphase = 0, l2phase = 0;
  uint32_t lphase[2] = {0u, 0u};
  bool pend[2] = {false, false};  // a stage copy into buffer b not yet seen complete
  bool pend2 = false;
  bool failed = false;
  // Z2 / P2 digit bytes of one shift
  const uint32_t zbytes = 7u * 128u * (uint32_t)cs * 2u;
  const uint32_t pbytes = 7u * (uint32_t)cs * (uint32_t)cs * 2u;
  const int kgz = cs / 8;

  // stage st of item (I, g) into buffer b: eight H digit tiles, seven P1 digit tiles
  auto stage_in = [&](int I, int g, int st, int b) {
    const uint32_t dst = sBase + (uint32_t)b * kStageBytes;
    const uint32_t lmb = lmb0 + 8u * (uint32_t)b;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lmb), "r"(kLoadBytes)
                 : "memory");
    for (int l = 0; l < kSDH; ++l)
      bulk_copy(dst + (uint32_t)(l * kAT * 2),
                a.Hs + BCK(((size_t)(l * a.RB + I) * a.KT + (JH0 + st)) * (kAT / 8), a.n_hs),
                (uint32_t)(kAT * 2), lmb);
    const size_t Pg0 = (size_t)g * kSD * kStages * kBT;
    for (int l = 0; l < kSD; ++l)
      bulk_copy(dst + (uint32_t)(kSDH * kAT * 2 + l * kBT * 2),
                a.Pd + BCK(Pg0 + ((size_t)l * kStages + st) * kBT, a.n_pd), (uint32_t)(kBT * 2), lmb);
  };
  // the group's Z2 digit tiles of row tile I, then its P2 digit tiles
  auto z2_in = [&](int I, int g, int nsh) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lmb2),
                 "r"((uint32_t)nsh * (zbytes + pbytes))
                 : "memory");
    for (int l = 0; l < nsh; ++l) {
      const int sh = g * S + l;
      bulk_copy(sBase + (uint32_t)l * zbytes, a.Zd + BCK(((size_t)sh * a.RB + I) * 7 * (128 * cs), a.n_zd),
                zbytes, lmb2);
      bulk_copy(sBase + (uint32_t)S * zbytes + (uint32_t)l * pbytes,
                a.P2d + BCK((size_t)sh * 7 * cs * cs, a.n_p2d), pbytes, lmb2);
    }
  };

  long long item = blockIdx.x;
  if (item < items) {
    pend[0] = true;
    if (tid == 0) stage_in((int)(item / G), (int)(item % G), 0, 0);
  }
  for (; item < items && !failed; item += gridDim.x) {
    const int I = (int)(item / G), g = (int)(item % G);
    const int nsh = min(S, a.s - g * S);  // shifts of this group
    // the group's sigma rows (and P2 for the double-float epilogue), column
    // exponents and shifts
    for (int e = tid; e < S * 2 * m * m; e += kUT) {
      const int l = e / (2 * m * m), o = e % (2 * m * m);
      const int sh = g * S + l;
      pcs[e] = sh < a.s ? a.pc[BCK((size_t)sh * 2 * kMaxM * kMaxM + o, a.n_pc)] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    for (int e = tid; e < S * cs; e += kUT) {
      const int l = e / cs, c = e % cs;
      const int sh = g * S + l;
      fexp[e] = (sh < a.s && c < 2 * m) ? a.pexp[(size_t)sh * 2 * kMaxM + c] : 0;
      if (TCZ) f2exp[e] = (sh < a.s) ? a.p2exp[(size_t)sh * 2 * kMaxM + c] : 0;
    }
    for (int l = tid; l < S; l += kUT) sig[l] = (g * S + l < a.s) ? a.shifts[g * S + l] : mkcd(0.0, 0.0);
    // ---- 1. Z1 P1: stage st in buffer st & 1
    for (int st = 0; st < nst; ++st) {
      const int buf = kBufU == 2 ? (st & 1) : 0;
      const bool lok = mbar_wait(lmb0 + 8u * (uint32_t)buf, lphase[buf], kUpdWait);
      if (__syncthreads_or(!lok)) {
        failed = true;
        break;
      }
      lphase[buf] ^= 1u;
      pend[buf] = false;
      const int iss = tid >> 5;
#if SSV_TCS_FUSED
      // fused levels: the P1 digit tiles sit side by side (kUN rows each, then
      // the zero tile), so one product of H digit kd against P1 digits
      // b0 .. b0 + c - 1 (N = kUN c <= 256) lands digit b in TMEM level kd + b;
      // the kd = 0 products cover every level and open the item, so one thread
      // issues all of them, and commits to every issuer barrier (their phases
      // stay in step with the Z2 P2 round)
      (void)iss;
      if (tid == 0) {
        fence_after();
        const uint32_t aBase = sBase + (uint32_t)buf * kStageBytes;
        const uint32_t bBase = aBase + (uint32_t)(kSDH * kAT * 2);
        constexpr uint32_t kSbo = (uint32_t)kKG * 128u;
        constexpr int kMaxC = 256 / kUN;
#pragma unroll
        for (int ks = 0; ks < kKS / 16; ++ks) {
#pragma unroll
          for (int kd = 0; kd < kSDH; ++kd) {
            const int nb = kd == 0 ? kLev : min(kSD, kLev - kd);  // P1 digits (7: the zero tile)
#pragma unroll
            for (int b0 = 0; b0 < nb; b0 += kMaxC) {
              const int c = min(kMaxC, nb - b0);
              const uint64_t ad = mat_desc(aBase + (uint32_t)(kd * kAT * 2 + ks * 256), 128u, kSbo);
              const uint64_t bd = mat_desc(bBase + (uint32_t)(b0 * kBT * 2 + ks * 256), 128u, kSbo);
              const bool first = st == 0 && ks == 0 && kd == 0;
              mma_bf16(tmem + (uint32_t)((kd + b0) * kUN), ad, bd, idesc_bf16(kUM, kUN * c), first ? 0u : 1u);
            }
          }
        }
        for (int q = 0; q < kIss; ++q) mma_commit(mb + 8u * (uint32_t)q);
      }
#else
      if ((tid & 31) == 0 && iss < kIss) {
        fence_after();
        const uint32_t aBase = sBase + (uint32_t)buf * kStageBytes;
        const uint32_t bBase = aBase + (uint32_t)(kSDH * kAT * 2);
        constexpr uint32_t kSbo = (uint32_t)kKG * 128u;
#pragma unroll 1
        for (int lv = 0; lv < kLev; ++lv) {
          if (level_owner(lv) != iss) continue;
#pragma unroll 1
          for (int kd = max(0, lv - (kSD - 1)); kd <= min(kSDH - 1, lv); ++kd) {
            const int ld = lv - kd;
#pragma unroll
            for (int ks = 0; ks < kKS / 16; ++ks) {
              const uint64_t ad = mat_desc(aBase + (uint32_t)(kd * kAT * 2 + ks * 256), 128u, kSbo);
              const uint64_t bd = mat_desc(bBase + (uint32_t)(ld * kBT * 2 + ks * 256), 128u, kSbo);
              const bool first = st == 0 && kd == max(0, lv - (kSD - 1)) && ks == 0;
              mma_bf16(tmem + (uint32_t)(lv * kUN), ad, bd, kIdescU, first ? 0u : 1u);
            }
          }
        }
        mma_commit(mb + 8u * (uint32_t)iss);
      }
#endif
      // the next stage streams into the other buffer, whose products finished
      // in the previous round (with one buffer: after these products)
      if (kBufU == 2 && st + 1 < nst) {
        pend[buf ^ 1] = true;
        if (tid == 0) stage_in(I, g, st + 1, buf ^ 1);
      }
      bool ok = true;
      for (int q = 0; q < kIss; ++q) ok = mbar_wait(mb + 8u * q, mphase, kUpdWait) && ok;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      mphase ^= 1u;
      if (kBufU == 1 && st + 1 < nst) {
        pend[0] = true;
        if (tid == 0) stage_in(I, g, st + 1, 0);
      }
    }
    if (failed) break;
    // both stage buffers are free: TCZ fetches the group's Z2 / P2 tiles into them
    if (TCZ) {
      pend2 = true;
      if (tid == 0) z2_in(I, g, nsh);
    }
    // ---- epilogue: thread (row, quarter) = (tid mod 128, tid / 128) takes one H
    //      row and 16 of the 64 columns; warps w, w + 4, w + 8, w + 12 read TMEM
    //      lanes 32 (w mod 4) ..
    fence_after();
    const int row = tid & (kUM - 1), qt = tid >> 7;
    const int ih = I * kUM + row;
    const bool live = ih < hrows;
    const int Ei = live ? a.hexp[BCK(ih, a.npad)] : 0;
    const int cdr = ih - j0;  // shifted-diagonal correction row of fresh column cdr
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(qt * 16);
    float4 acc[8];
    bool ok_j[8];
    {
      float ah[16], al[16];
      drain_levels(tl, kLev, ah, al);
      // slot j (0 .. 7) of this quarter = group columns col, col + 1 with
      // col = 16 qt + 2 j: shift l = col / cs, complex column q = (col mod cs) / 2
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = qt * 16 + 2 * j, l = col / cs, q = (col % cs) >> 1;
        ok_j[j] = live && q < m && l < S && g * S + l < a.s;
        acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok_j[j]) {
          const int er = fexp[col], ei = fexp[col + 1];
          if (Ei == kBadExp || er == kBadExp || ei == kBadExp) {
            acc[j] = make_float4(__int_as_float(0x7fc00000), 0.f, __int_as_float(0x7fc00000), 0.f);
          } else {
            acc[j] = make_float4(ldexpf(ah[2 * j], Ei + er), ldexpf(al[2 * j], Ei + er),
                                 ldexpf(ah[2 * j + 1], Ei + ei), ldexpf(al[2 * j + 1], Ei + ei));
          }
        }
      }
    }
    if (TCZ) {
      // ---- 2. Z2 P2: the levels of Z1 P1 are read; the same TMEM columns take
      //      the seven levels of the group's Z2 digit tiles x P2 digit tiles
      fence_before();
      __syncthreads();
      const bool lok = mbar_wait(lmb2, l2phase, kUpdWait);
      if (__syncthreads_or(!lok)) {
        failed = true;
        break;
      }
      l2phase ^= 1u;
      pend2 = false;
      const int iss = tid >> 5;
#if SSV_TCS_FUSED
      // fused levels: shift l's seven levels sit side by side in TMEM (columns
      // 7 cs l + cs lv) and its P2 digit tiles (cs rows each) are stacked, so one
      // product of Z2 digit kd against P2 digits 0 .. 6 - kd (N = cs (7 - kd))
      // lands digit ld in level kd + ld; kd = 0 opens all seven
      (void)iss;
      if (tid == 0) {
        fence_after();
        const uint32_t sboz = (uint32_t)kgz * 128u;
        for (int l = 0; l < nsh; ++l) {
          const uint32_t zb = sBase + (uint32_t)l * zbytes;
          const uint32_t pb = sBase + (uint32_t)S * zbytes + (uint32_t)l * pbytes;
#pragma unroll 1
          for (int ks = 0; ks < cs / 16; ++ks) {
#pragma unroll
            for (int kd = 0; kd < 7; ++kd) {
              const uint64_t ad = mat_desc(zb + (uint32_t)(kd * 128 * cs * 2 + ks * 256), 128u, sboz);
              const uint64_t bd = mat_desc(pb + (uint32_t)(ks * 256), 128u, sboz);
              mma_bf16(tmem + (uint32_t)(7 * cs * l + kd * cs), ad, bd, idesc_bf16(kUM, cs * (7 - kd)),
                       (kd == 0 && ks == 0) ? 0u : 1u);
            }
          }
        }
        for (int q = 0; q < kIss; ++q) mma_commit(mb + 8u * (uint32_t)q);
      }
#else
      if ((tid & 31) == 0 && iss < kIss) {
        fence_after();
        const uint32_t idz = idesc_bf16(kUM, cs);
        const uint32_t sboz = (uint32_t)kgz * 128u;
#pragma unroll 1
        for (int lv = 0; lv < 7; ++lv) {
          if (level_owner(lv) != iss) continue;
#pragma unroll 1
          for (int l = 0; l < nsh; ++l) {
            const uint32_t zb = sBase + (uint32_t)l * zbytes;
            const uint32_t pb = sBase + (uint32_t)S * zbytes + (uint32_t)l * pbytes;
#pragma unroll 1
            for (int kd = 0; kd <= lv; ++kd) {
              const int ld = lv - kd;
#pragma unroll 1
              for (int ks = 0; ks < cs / 16; ++ks) {
                const uint64_t ad = mat_desc(zb + (uint32_t)(kd * 128 * cs * 2 + ks * 256), 128u, sboz);
                const uint64_t bd = mat_desc(pb + (uint32_t)(ld * cs * cs * 2 + ks * 256), 128u, sboz);
                mma_bf16(tmem + (uint32_t)(lv * kUN + l * cs), ad, bd, idz, (kd == 0 && ks == 0) ? 0u : 1u);
              }
            }
          }
        }
        mma_commit(mb + 8u * (uint32_t)iss);
      }
#endif
      bool ok = true;
      for (int q = 0; q < kIss; ++q) ok = mbar_wait(mb + 8u * q, mphase, kUpdWait) && ok;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      mphase ^= 1u;
      // the Z2 / P2 tiles covered buffer 0's zero tile: write it again before
      // the next item's first products read it (ordered by the load wait and
      // barrier that precede them)
      for (int b = 0; b < kBufU; ++b)
        if ((size_t)b * kStageBytes + kZeroOff < (size_t)S * (zbytes + pbytes)) zero_tile(b);
    }
    // ---- 3. the stage buffers are free again: the next item's first stage
    //      streams in during the rest of the epilogue
    if (item + gridDim.x < items) {
      const long long nx = item + gridDim.x;
      pend[0] = true;
      if (tid == 0) stage_in((int)(nx / G), (int)(nx % G), 0, 0);
    }
    if (TCZ) {
      fence_after();
      float ah[16], al[16];
#if SSV_TCS_FUSED
      // shift l = (16 qt) / cs: its levels start at column 7 cs l, this
      // quarter's columns at (16 qt) mod cs within them
      drain_levels(tl - (uint32_t)(qt * 16) + (uint32_t)(7 * cs * ((qt * 16) / cs) + (qt * 16) % cs), 7, ah, al,
                   cs);
#else
      drain_levels(tl, 7, ah, al);
#endif
      const int l = (qt * 16) / cs;  // one shift per quarter (cs >= 16)
      const int sh = g * S + l;
      const int Ez = (live && sh < a.s) ? a.zexp[BCK((size_t)sh * a.npad + ih, (size_t)a.s * a.npad)] : 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (!ok_j[j]) continue;
        const int col = qt * 16 + 2 * j;
        const int fr = f2exp[col], fi = f2exp[col + 1];
        if (Ez == kBadExp || fr == kBadExp || fi == kBadExp) {
          acc[j] = make_float4(__int_as_float(0x7fc00000), 0.f, __int_as_float(0x7fc00000), 0.f);
          continue;
        }
        // acc += level sum, both double-float: two-sum of the high words
        auto addpair = [](float& h, float& lo, float bh, float bl) {
          const float s2 = h + bh;
          const float bp = s2 - h;
          lo += ((h - (s2 - bp)) + (bh - bp)) + bl;
          h = s2;
        };
        addpair(acc[j].x, acc[j].y, ldexpf(ah[2 * j], Ez + fr), ldexpf(al[2 * j], Ez + fr));
        addpair(acc[j].z, acc[j].w, ldexpf(ah[2 * j + 1], Ez + fi), ldexpf(al[2 * j + 1], Ez + fi));
      }
    } else if (live) {
      // several shifts per quarter (m <= 4): + Z2(row, :) P2(:, q) in
      // double-float from the old row of each slot's shift
#pragma unroll 1
      for (int qq = 0; qq < m; ++qq) {
        int lz = -1;
        float4 zz = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (!ok_j[j]) continue;
          const int col = qt * 16 + 2 * j, l = col / cs, q = (col % cs) >> 1;
          if (l != lz) {
            zz = a.Z2[BCK((size_t)(g * S + l) * a.z2_stride + (p + ih) + (size_t)qq * ldz, a.n_z2)];
            lz = l;
          }
          const float4 w = pcs[(size_t)l * 2 * m * m + qq * m + q];
          df_mac(acc[j].x, acc[j].y, zz.x, zz.y, w.x, w.y);
          df_mac(acc[j].x, acc[j].y, -zz.z, -zz.w, w.z, w.w);
          df_mac(acc[j].z, acc[j].w, zz.x, zz.y, w.z, w.w);
          df_mac(acc[j].z, acc[j].w, zz.z, zz.w, w.x, w.y);
        }
      }
    }
    if (live && cdr >= 0 && cdr < nsig) {
      // - sigma P1(cdr, q)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (!ok_j[j]) continue;
        const int col = qt * 16 + 2 * j, l = col / cs, q = (col % cs) >> 1;
        const float4 sgf = df_split(sig[l]);
        const float4 w = pcs[(size_t)l * 2 * m * m + m * m + cdr * m + q];
        df_mac(acc[j].x, acc[j].y, -sgf.x, -sgf.y, w.x, w.y);
        df_mac(acc[j].x, acc[j].y, sgf.z, sgf.w, w.z, w.w);
        df_mac(acc[j].z, acc[j].w, -sgf.x, -sgf.y, w.z, w.w);
        df_mac(acc[j].z, acc[j].w, -sgf.z, -sgf.w, w.x, w.y);
      }
    }
    // normalised pairs
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float sr = acc[j].x + acc[j].y, si = acc[j].z + acc[j].w;
      acc[j] = make_float4(sr, acc[j].y - (sr - acc[j].x), si, acc[j].w - (si - acc[j].z));
    }
    float mx = 0.f;
    if (TCZ) {
      // the new row's digit exponent: the maximum over the shift's 2m entries,
      // which two quarters share when cs = 32
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (!ok_j[j]) continue;
        mx = fmaxf(mx, fmaxf(fabsf(acc[j].x), fabsf(acc[j].z)));
        if (!(fabsf(acc[j].x) <= 3.4e38f) || !(fabsf(acc[j].z) <= 3.4e38f)) mx = __int_as_float(0x7f800000);
      }
      xmax[qt * kUM + row] = mx;
    }
    // a shift's row may be shared by two quarters: every old entry (double-float
    // path) and every maximum is read before the writes below
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (!ok_j[j]) continue;
      const int col = qt * 16 + 2 * j, l = col / cs, q = (col % cs) >> 1;
      a.Z2[BCK((size_t)(g * S + l) * a.z2_stride + (p + ih) + (size_t)q * ldz, a.n_z2)] = acc[j];
    }
    if (TCZ && live) {
      const int l = (qt * 16) / cs, sh = g * S + l;
      if (sh < a.s) {
        if (cs == 32) mx = fmaxf(mx, xmax[(qt ^ 1) * kUM + row]);
        const int E = scale_exp_f(mx);
        const int kb = (qt * 16) % cs;  // this quarter's first K entry of the row
        if ((qt * 16) % cs == 0) a.zexp[BCK((size_t)sh * a.npad + ih, (size_t)a.s * a.npad)] = E;
        const size_t T0 = ((size_t)sh * a.RB + I) * 7 * (128 * cs);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          unsigned short dg[8][7];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = h * 4 + (e >> 1);
            const bool use = ok_j[j];
            const float hi = use ? ((e & 1) ? acc[j].z : acc[j].x) : 0.f;
            const float lo = use ? ((e & 1) ? acc[j].w : acc[j].y) : 0.f;
            digits7_pair(hi, lo, E, dg[e]);
          }
          const int off = tile_off_kg(row, kb + h * 8, kgz);
#pragma unroll
          for (int l2 = 0; l2 < 7; ++l2) {
            uint4 u;
            u.x = dg[0][l2] | ((unsigned)dg[1][l2] << 16);
            u.y = dg[2][l2] | ((unsigned)dg[3][l2] << 16);
            u.z = dg[4][l2] | ((unsigned)dg[5][l2] << 16);
            u.w = dg[6][l2] | ((unsigned)dg[7][l2] << 16);
            *reinterpret_cast<uint4*>(a.Zd + BCK(T0 + (size_t)l2 * (128 * cs) + off, a.n_zd)) = u;
          }
        }
      }
    }
    fence_before();
    __syncthreads();
  }
  if (failed) {
    // a completion never arrived: record it, give the products and copies in
    // flight one more bounded wait, then release TMEM
    if (tid == 0) {
      atomicExch(a.err, 1);
      for (int q = 0; q < kIss; ++q) mbar_wait(mb + 8u * q, mphase, kUpdWait);
      for (int b = 0; b < 2; ++b)
        if (pend[b]) mbar_wait(lmb0 + 8u * (uint32_t)b, lphase[b], kUpdWait);
      if (pend2) mbar_wait(lmb2, l2phase, kUpdWait);
    }
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

#ifdef SSV_BOUNDS_CHECK
// bit 2 of the error word when a byte of the canary after the scratch changed
__global__ void tcs_canary_kernel(const unsigned char* c, size_t nbytes, int* err) {
  for (size_t i = threadIdx.x; i < nbytes; i += blockDim.x)
    if (c[i] != 0xA5) atomicOr(err, 4);
}
#endif

// ---- final m x m block, G or the X-hat back pass ----------------------------
__global__ void __launch_bounds__(kPT) tcs_final_kernel(TcsArgs a, int nsteps, int nbe_first) {
  __shared__ cd Wm[kMaxM * 2 * kMaxM];
  __shared__ cd lmul[kMaxM];
  __shared__ cd Yb[kMaxM * kMaxM];
  __shared__ cd zs[kMaxM * kMaxM], p2s[kMaxM * kMaxM], zn[kMaxM * kMaxM];
  __shared__ int s_piv, s_sing;
  const int sh = blockIdx.x, tid = threadIdx.x;
  const int n = a.n, m = a.m, p = a.p, ldz = p + n;
  const cd sigma = a.shifts[sh];
  const double sing_tol = (double)n * 7.105427357601002e-15 * sqrt(shifted_norm2(a.hnorm, n, sigma));
  const float4* Z2f = a.Z2 + (size_t)sh * a.z2_stride;
  const bool failed = *a.err != 0;
  if (tid == 0) s_sing = a.flags[sh];
  for (int idx = tid; idx < m * 2 * m; idx += kPT) {
    const int i = idx % m, j = idx / m;
    cd v;
    if (j < m) v = df_join(Z2f[BCK((p + i) + (size_t)j * ldz, a.z2_stride)]);
    else v = mkcd(i <= j - m ? a.R[i + (size_t)(j - m) * n] : 0.0, 0.0);
    Wm[i + j * kMaxM] = v;
  }
  __syncthreads();
  // Gauss-Jordan with partial pivoting on [Wm | R(0:m, 0:m)]
  for (int kk = 0; kk < m; ++kk) {
    if (tid < 32) {
      double best = -1.0;
      int brow = kk;
      for (int i = kk + tid; i < m; i += 32) {
        const double v = cabs1(Wm[i + kk * kMaxM]);
        if (v > best) { best = v; brow = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int orow = __shfl_xor_sync(0xffffffffu, brow, o);
        if (ob > best || (ob == best && orow < brow)) { best = ob; brow = orow; }
      }
      if (tid == 0) {
        s_piv = brow;
        const cd pv = Wm[brow + kk * kMaxM];
        if (best == 0.0 || sqrt(pv.x * pv.x + pv.y * pv.y) <= sing_tol) s_sing = 1;
      }
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != kk) {
      for (int j = tid; j < 2 * m; j += kPT) {
        const cd t = Wm[kk + j * kMaxM];
        Wm[kk + j * kMaxM] = Wm[pr + j * kMaxM];
        Wm[pr + j * kMaxM] = t;
      }
    }
    __syncthreads();
    const cd d = Wm[kk + kk * kMaxM];
    const bool dz = (d.x == 0.0 && d.y == 0.0);
    if (tid < m) lmul[tid] = (tid == kk || dz) ? mkcd(0.0, 0.0) : cdiv(Wm[tid + kk * kMaxM], d);
    __syncthreads();
    for (int idx = tid; idx < m * 2 * m; idx += kPT) {
      const int i = idx % m, j = idx / m;
      if (i != kk && j > kk) Wm[i + j * kMaxM] = cfms(lmul[i], Wm[kk + j * kMaxM], Wm[i + j * kMaxM]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < m * m; idx += kPT) {
    const int i = idx % m, q = idx / m;
    const cd d = Wm[i + i * kMaxM];
    Yb[i + q * kMaxM] = (d.x == 0.0 && d.y == 0.0) ? mkcd(0.0, 0.0) : cdiv(Wm[i + (m + q) * kMaxM], d);
  }
  __syncthreads();
  const bool sing = s_sing != 0;
  const double nanv = __longlong_as_double(0x7ff8000000000000LL);
  const bool bad = sing || failed;
  cd* tout = a.out + (size_t)sh * m * a.ldo;
  if (a.mode == SSV_G || a.mode == SSV_TF) {
    const double sgn = a.mode == SSV_TF ? -1.0 : 1.0;
    for (int idx = tid; idx < p * m; idx += kPT) {
      const int i = idx % p, q = idx / p;
      cd acc = mkcd(0.0, 0.0);
      for (int t = 0; t < m; ++t)
        acc = cfma(df_join(Z2f[BCK(i + (size_t)t * ldz, a.z2_stride)]), Yb[t + q * kMaxM], acc);
      if (bad) acc = mkcd(nanv, nanv);
      tout[BCK(i, p) + (size_t)q * a.ldo] = mkcd(sgn * acc.x, sgn * acc.y);
    }
  } else {
    // backward pass: z = Y; per step b = B .. 1: X-hat rows of b = P1_b z,
    // then z = P2_b z; the initial live rows n - m .. n - 1 take the last z.
    // Step b covers the fresh columns j0_b = (B - b) n_b .. + nbe_b - 1.
    const cd* ZT = a.ZT + (size_t)sh * (size_t)n * m;
    for (int e = tid; e < m * m; e += kPT) zs[(e % m) + (e / m) * kMaxM] = Yb[(e % m) + (e / m) * kMaxM];
    __syncthreads();
    for (int b = nsteps; b >= 1; --b) {
      const int nbe_b = b == 1 ? nbe_first : kNBT;
      const int j0b = (nsteps - b) * kNBT;
      for (int e = tid; e < m * m; e += kPT)
        p2s[(e % m) + (e / m) * kMaxM] = tout[BCK(n - b * m + e % m, n) + (size_t)(e / m) * a.ldo];
      __syncthreads();
      for (int idx = tid; idx < nbe_b * m; idx += kPT) {
        const int i = j0b + idx % nbe_b, q = idx / nbe_b;
        cd acc = mkcd(0.0, 0.0);
        for (int t = 0; t < m; ++t) acc = cfma(ZT[BCK(i + (size_t)t * n, (size_t)n * m)], zs[t + q * kMaxM], acc);
        tout[BCK(i, n) + (size_t)q * a.ldo] = bad ? mkcd(nanv, nanv) : acc;
      }
      for (int e = tid; e < m * m; e += kPT) {
        const int rr = e % m, q = e / m;
        cd acc = mkcd(0.0, 0.0);
        for (int t = 0; t < m; ++t) acc = cfma(p2s[rr + t * kMaxM], zs[t + q * kMaxM], acc);
        zn[rr + q * kMaxM] = acc;
      }
      __syncthreads();
      for (int e = tid; e < m * m; e += kPT) zs[(e % m) + (e / m) * kMaxM] = zn[(e % m) + (e / m) * kMaxM];
      __syncthreads();
    }
    for (int e = tid; e < m * m; e += kPT) {
      const int rr = e % m, q = e / m;
      tout[(n - m + rr) + (size_t)q * a.ldo] = bad ? mkcd(nanv, nanv) : zs[rr + q * kMaxM];
    }
  }
  if (a.status != nullptr && tid == 0) {
    bool fin = true;
    for (int e = 0; e < m * m; ++e) {
      const cd y = Yb[(e % m) + (e / m) * kMaxM];
      fin = fin && isfinite(y.x) && isfinite(y.y);
    }
    a.status[sh] = sing ? SSV_SHIFT_SINGULAR : ((fin && !failed) ? SSV_SHIFT_OK : SSV_SHIFT_NONFINITE);
  }
}

}  // namespace

bool solve_tc_supported(const Handle* h, int mode) {
  return h->m <= kMaxM && h->n > h->m && (mode == SSV_G || mode == SSV_TF || mode == SSV_XHAT);
}

size_t solve_tc_scratch_bytes(int n, int m, int p, int s, int mode) {
  const int cs = shift_cols(m), S = kUN / cs;
  const size_t G = (size_t)(s + S - 1) / S;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  size_t b = al(sizeof(float4) * (size_t)s * (size_t)(p + n) * m);
  if (mode == SSV_XHAT) b += al(sizeof(cd) * (size_t)s * (size_t)n * m);
  b += al(G * kSD * kStages * kBT * 2) + al(sizeof(int) * (size_t)s * 2 * kMaxM) +
       al(sizeof(float4) * (size_t)s * 2 * kMaxM * kMaxM) + al(sizeof(int) * ((size_t)s + 1));
  if (cs >= 16) {  // Z2 P2 on the tensor cores: window and P2 digit tiles
    const size_t np = (size_t)resid_tc_npad(n);
    b += al((size_t)s * np * 7 * cs * 2) + al(sizeof(int) * (size_t)s * np) +
         al((size_t)s * 7 * cs * cs * 2) + al(sizeof(int) * (size_t)s * 2 * kMaxM);
  }
  return b + 256;
}

int solve_tc(const Handle* h, int s, const double* shifts, int mode, double* out, long long ldo,
             int* status, const void* hdig, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  if (!solve_tc_supported(h, mode)) return SSV_ENOTSUP;
  if (resid_tc_ktile() != kKS) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  const int cs = shift_cols(m), S = kUN / cs;
  const int G = (s + S - 1) / S;
  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t bZ = al(sizeof(float4) * (size_t)s * (size_t)(p + n) * m);
  const size_t bT = mode == SSV_XHAT ? al(sizeof(cd) * (size_t)s * (size_t)n * m) : 0;
  const size_t bP = al((size_t)G * kSD * kStages * kBT * 2);
  const size_t bE = al(sizeof(int) * (size_t)s * 2 * kMaxM);
  const size_t bC = al(sizeof(float4) * (size_t)s * 2 * kMaxM * kMaxM);
  const size_t bF = al(sizeof(int) * ((size_t)s + 1));
  const size_t bH = hdig == nullptr ? al(resid_tc_hbytes(n)) : 0;
  const int np = resid_tc_npad(n);
  const bool tcz = cs >= 16;
  const size_t bZd = tcz ? al((size_t)s * np * 7 * cs * 2) : 0;
  const size_t bZe = tcz ? al(sizeof(int) * (size_t)s * np) : 0;
  const size_t bPd2 = tcz ? al((size_t)s * 7 * cs * cs * 2) : 0;
  const size_t bPe2 = tcz ? al(sizeof(int) * (size_t)s * 2 * kMaxM) : 0;
  const size_t total = bZ + bT + bP + bE + bC + bF + bZd + bZe + bPd2 + bPe2 + bH;
#ifdef SSV_BOUNDS_CHECK
  constexpr size_t kCanary = 256;  // checked after the last block step
#else
  constexpr size_t kCanary = 0;
#endif
  unsigned char* buf = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&buf, total + kCanary, st));
  unsigned char* o = buf;
  TcsArgs a;
  a.n = n; a.m = m; a.p = p; a.s = s; a.cs = cs; a.S = S; a.ngroups = G; a.mode = mode;
  a.H = h->H; a.Hhi = h->Hhi; a.Hlo = h->Hlo; a.Ct = h->Ct; a.ldct = p > 0 ? p : 1; a.R = h->R;
  a.shifts = reinterpret_cast<const cd*>(shifts); a.hnorm = h->hnorm2;
  a.Z2 = reinterpret_cast<float4*>(o); o += bZ;
  a.z2_stride = (size_t)(p + n) * m;
  a.ZT = bT ? reinterpret_cast<cd*>(o) : nullptr; o += bT;
  a.Pd = reinterpret_cast<uint16_t*>(o); o += bP;
  a.pexp = reinterpret_cast<int*>(o); o += bE;
  a.pc = reinterpret_cast<float4*>(o); o += bC;
  a.flags = reinterpret_cast<int*>(o);
  a.err = a.flags + s; o += bF;
  a.tcz = tcz ? 1 : 0;
  a.npad = np;
  a.Zd = tcz ? reinterpret_cast<uint16_t*>(o) : nullptr; o += bZd;
  a.zexp = tcz ? reinterpret_cast<int*>(o) : nullptr; o += bZe;
  a.P2d = tcz ? reinterpret_cast<uint16_t*>(o) : nullptr; o += bPd2;
  a.p2exp = tcz ? reinterpret_cast<int*>(o) : nullptr; o += bPe2;
  a.out = reinterpret_cast<cd*>(out); a.ldo = ldo; a.status = status;
  a.RB = np / kUM;
  a.KT = np / kKS;
  a.n_z2 = (size_t)s * a.z2_stride;
  a.n_zt = bT ? (size_t)s * n * m : 0;
  a.n_pd = (size_t)G * kSD * kStages * kBT;
  a.n_zd = tcz ? (size_t)s * np * 7 * cs : 0;
  a.n_p2d = tcz ? (size_t)s * 7 * cs * cs : 0;
  a.n_pc = (size_t)s * 2 * kMaxM * kMaxM;
  a.n_hs = (size_t)np * np;  // uint4 of the eight H digit slices
  a.n_out = 0;
  int rc = SSV_OK;
  cudaError_t e = cudaSuccess;
#ifdef SSV_BOUNDS_CHECK
  // scratch read before it is written shows up as NaN (0xFF bytes), and the
  // canary after the scratch as a changed byte
  e = cudaMemsetAsync(buf, 0xFF, total, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf + total, 0xA5, kCanary, st);
#endif
  if (e == cudaSuccess) e = cudaMemsetAsync(a.Pd, 0, bP, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.err, 0, sizeof(int), st);
  if (e == cudaSuccess && hdig == nullptr) {
    rc = resid_tc_split_h(h, o, st);
    hdig = o;
  }
  if (e == cudaSuccess && rc == SSV_OK) {
    const unsigned char* hb = static_cast<const unsigned char*>(hdig);
    a.Hs = reinterpret_cast<const uint4*>(hb);
    a.hexp = reinterpret_cast<const int*>(hb + ((size_t)kDigits * np * np * 2 + 255) / 256 * 256);
    const size_t psm = sizeof(PanelSmem);
    e = cudaFuncSetAttribute(tcs_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm);
    // three panels per SM (74 KB of shared memory each)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tcs_panel_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tcs_update_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kUpdSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(tcs_update_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kUpdSmem);
    if (e == cudaSuccess) {
      tcs_setup_kernel<<<s, kPT, 0, st>>>(a);
      count_launch();
      int nbe_first = (n - m) % kNBT;
      if (nbe_first == 0) nbe_first = kNBT;
      int k = n, step = 0;
      while (k > m) {
        const int nbe = step == 0 ? nbe_first : kNBT;
        ++step;
        tcs_panel_kernel<<<s, kPT, psm, st>>>(a, k, nbe, step);
        count_launch();
        const int hrows = k - nbe;
        if (hrows > 0) {
          const long long items = (long long)((hrows + kUM - 1) / kUM) * G;
          const int grid =
              (int)std::max<long long>(1, std::min<long long>(items, (long long)num_sms() * kCtasU));
          void* tru = trace_begin("tcs_update", st);  // per-launch span when tracing is on
          if (tcz) tcs_update_kernel<true><<<grid, kUT, kUpdSmem, st>>>(a, k, nbe);
          else tcs_update_kernel<false><<<grid, kUT, kUpdSmem, st>>>(a, k, nbe);
          count_launch();
          trace_end(tru, st);
        }
        k -= nbe;
      }
#ifdef SSV_BOUNDS_CHECK
      tcs_canary_kernel<<<1, 256, 0, st>>>(buf + total, kCanary, a.err);
      count_launch();
#endif
      tcs_final_kernel<<<s, kPT, 0, st>>>(a, step, nbe_first);
      count_launch();
      e = cudaGetLastError();
    }
  }
  if (e != cudaSuccess) {
    set_cuda_error(e);
    rc = SSV_ECUDA;
  }
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (e2 != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e2);
    rc = SSV_ECUDA;
  }
  return rc;
}

}  // namespace ssv
