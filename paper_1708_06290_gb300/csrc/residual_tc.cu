// FP64-accurate residual E = R - (H - sigma I) Xhat on the tensor cores.
//
// The certification step of the mixed path (the refinement residual of
// iterative refinement; the residual of Sec. 3.3's unreduced right-hand-side
// technique) needs H Xhat to about 2^-50 of ||H|| ||Xhat||.  It is formed by
// error-free splitting (Ozaki, Ogita, Oishi, Rump 2012):
//
//   * each row i of H (its structural part, columns j >= i - m) is written as
//     H(i, j) = (-1)^s 2^{E_i} sum_{k=1..8} d_k 2^{-7k}, d_k in [0, 127],
//     with 2^{E_i} > max_j |H(i, j)|, and likewise each real column c of Xhat
//     (Re and Im of every column q) with its own exponent E_c;
//   * the digits are exact in BF16, so every slice product H_k X_l is exact in
//     FP32 as long as each partial sum stays below 2^24: with windows of 128
//     terms and the (t - 1) products of one level t = k + l summed together,
//     |sum| <= 8 * 128 * 127^2 < 2^24;
//   * H X = 2^{E_i + E_c} sum_{t=2..9} 2^{-7t} L_t, L_t = sum_{k+l=t} H_k X_l
//     (the 36 products with k + l <= 9; the dropped ones are below
//     2^{-56} relative to the row and column scales).
//
// Persistent CTAs (two per SM) take work items of 128 rows of H and one
// shift (N = 32 real columns, 2m of them live).  Per 32-deep K stage the
// sixteen slice tiles (no-swizzle K-major core-matrix layout, stored tile by
// tile in global memory) are copied into shared memory by one thread with
// 1-D TMA bulk copies completing on an mbarrier; four threads (lane 0 of each warp, each owning two of
// the eight levels) issue the 72 tcgen05.mma (kind::f16, BF16 x BF16 -> FP32,
// M = 128, N = 32, K = 16) into eight TMEM accumulators (one per level, 32
// columns each) and commit to their own mbarriers; after every fourth stage
// the warps read the levels back (tcgen05.ld) and add them, scaled by
// 2^{-7t}, into double-float accumulators.  The epilogue forms E in FP64.
#include <algorithm>

#include "ssv_internal.cuh"
#include "tc_common.cuh"

namespace ssv {

namespace {

constexpr int kM = 128;       // rows of H per tile = TMEM lanes
constexpr int kN = 32;        // real columns per shift (2m, zero-padded)
// Tile-shape parameters.  Measured on GB300 at n = 5000, m = 16 (ms per 2000
// shifts): the products are small (N = 32), so throughput follows the number
// of threads issuing them: one CTA per SM with two TMEM windows and the next
// stage prefetched 208; two CTAs per SM, 16-deep stages, prefetched 142; two
// CTAs per SM, 32-deep stages, one buffer 128, with two issuers 122, with four
// 112, and staged by TMA bulk copies instead of cp.async 106 (the default);
// without the products at all 61 (staging by cp.async, and readout).  TMA bulk
// copies into two buffers: 16-deep stages, two CTAs per SM 136; 32-deep
// stages, one CTA per SM with two TMEM windows 152 (the N = 32 products, not
// the copies, set the pace).
#ifndef SSV_TC_KS
#define SSV_TC_KS 32          // K per shared-memory stage (16 or 32)
#endif
#ifndef SSV_TC_TWO_WINDOWS
#define SSV_TC_TWO_WINDOWS 0  // 1: two TMEM windows in flight, one CTA per SM
#endif
#ifndef SSV_TC_INTERLEAVE
#define SSV_TC_INTERLEAVE 0   // 1: consecutive products to different levels (one issuer)
#endif
#ifndef SSV_TC_ISSUERS
#define SSV_TC_ISSUERS 4      // threads issuing products, each owning whole levels
#endif
#ifndef SSV_TC_BUFFERS
#define SSV_TC_BUFFERS 1      // 2: the next stage streams in during the products
#endif
#ifndef SSV_TC_FUSED
#define SSV_TC_FUSED 1        // 1: fused-level products in the two-shift kernel (24 per stage)
#endif
#ifndef SSV_TC_PAIRS
#define SSV_TC_PAIRS 1        // 1: two shifts per work item (N = 64, one CTA per SM)
#endif
#ifndef SSV_TC_BULK
#define SSV_TC_BULK 1         // one buffer: stage with 1-D TMA bulk copies (else cp.async)
#endif
constexpr int kKS = SSV_TC_KS;  // K per shared-memory stage (16 or 32)
constexpr bool kPairs = SSV_TC_PAIRS != 0;
constexpr int kSl = 8;        // digit slices of H and of Xhat
constexpr int kLev = 8;       // levels t = 2 .. 9
constexpr int kWin = 128 / kKS;  // stages per exact accumulation window (K = 128)
constexpr int kKG = kKS / 8;     // core matrices along K in a tile
constexpr int kAT = kM * kKS;    // BF16 elements of one H slice tile
constexpr int kBT = kN * kKS;    // BF16 elements of one Xhat slice tile
// two accumulation windows in flight (the finished one is read while the next
// multiplies: all of TMEM, one CTA per SM) or one (two CTAs per SM)
constexpr bool kTwoWin = SSV_TC_TWO_WINDOWS != 0;
constexpr int kTmemCols = (kTwoWin ? 2 : 1) * kLev * kN;
constexpr int kCtasPerSm = kTwoWin ? 1 : 2;
constexpr uint32_t kStageBytes = (uint32_t)kSl * (kAT + kBT) * 2;
constexpr int kBuf = SSV_TC_BUFFERS;  // 2: the next stage streams in during the products
constexpr int kIss = SSV_TC_ISSUERS;  // threads issuing products (lane 0 of warps 0 ..)
constexpr bool kBulk = SSV_TC_BULK != 0;
static_assert(kIss == 1 || kIss == 2 || kIss == 4, "issuers");
constexpr size_t kSmem = kBuf * (size_t)kStageBytes + 64;
static_assert(kCtasPerSm * kSmem <= 227 * 1024, "shared memory of the resident CTAs");
static_assert(kCtasPerSm * kTmemCols <= 512, "TMEM columns of the resident CTAs");
using namespace tcg;
constexpr uint32_t kIdesc = idesc_bf16(kM, kN);
static_assert(kSl == kDigits, "eight digit slices");

// element offset inside a K-major core-matrix tile with kKG core matrices
// along K: core (row group g, K group kk) at (g * kKG + kk) * 64 elements,
// 8 rows of 8 contiguous elements each (byte strides: 128 along K, kKG * 128
// along rows)
__host__ __device__ __forceinline__ int tile_off(int row, int k) {
  return (((row >> 3) * kKG + (k >> 3)) * 8 + (row & 7)) * 8 + (k & 7);
}

__global__ void tc_hrow_kernel(int n, int m, int npad, const double* __restrict__ H,
                               int* __restrict__ hexp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i >= n) {
    hexp[i] = 0;
    return;
  }
  double mx = 0.0;
  bool bad = false;
  for (int j = max(0, i - m); j < n; ++j) {
    const double v = fabs(H[i + (size_t)j * n]);
    if (!(v <= 1.7976931348623157e308)) bad = true;
    else mx = fmax(mx, v);
  }
  hexp[i] = bad ? kBadExp : scale_exp(mx);
}

// items (i, j8): rows i fastest (coalesced reads of column-major H)
__global__ void tc_hsplit_kernel(int n, int m, int npad, const double* __restrict__ H,
                                 const int* __restrict__ hexp, uint4* __restrict__ Hs) {
  const int KT = npad / kKS, RB = npad / kM;
  const long long items = (long long)npad * (npad / 8);
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(it % npad), j8 = (int)(it / npad);
    const int E = hexp[i];
    unsigned short dg[8][kSl];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = j8 * 8 + e;
      const double v = (i < n && j < n && j >= i - m) ? H[i + (size_t)j * n] : 0.0;
      digits8(v, E, dg[e]);
    }
    const int I = i / kM, J = (j8 * 8) / kKS;
    const int off = tile_off(i % kM, (j8 * 8) % kKS);
#pragma unroll
    for (int l = 0; l < kSl; ++l) {
      uint4 w;
      w.x = dg[0][l] | ((unsigned)dg[1][l] << 16);
      w.y = dg[2][l] | ((unsigned)dg[3][l] << 16);
      w.z = dg[4][l] | ((unsigned)dg[5][l] << 16);
      w.w = dg[6][l] | ((unsigned)dg[7][l] << 16);
      const size_t base = ((size_t)(l * RB + I) * KT + J) * kAT + off;
      Hs[base / 8] = w;
    }
  }
}

// one block per active shift: column exponents, then the digit tiles
__global__ void __launch_bounds__(256) tc_xsplit_kernel(int n, int m, int npad,
                                                        const int* __restrict__ list,
                                                        const int* __restrict__ count,
                                                        const cd* __restrict__ X, long long ldx,
                                                        uint4* __restrict__ Xs,
                                                        int* __restrict__ xexp) {
  const int w = blockIdx.x;
  if (w >= *count) return;
  const int sh = list[w];
  const int tid = threadIdx.x;
  const int KT = npad / kKS;
  const cd* Xh = X + (size_t)sh * m * ldx;
  __shared__ int sE[kN];
  {
    const int c = tid >> 3, part = tid & 7;  // 8 threads per real column
    double mx = 0.0;
    bool bad = false;
    if (c < 2 * m) {
      const int q = c >> 1;
      for (int j = part; j < n; j += 8) {
        const cd x = Xh[j + (size_t)q * ldx];
        const double v = fabs((c & 1) ? x.y : x.x);
        if (!(v <= 1.7976931348623157e308)) bad = true;
        else mx = fmax(mx, v);
      }
    }
    for (int o = 4; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      bad = __shfl_xor_sync(0xffffffffu, (int)bad, o) || bad;
    }
    if (part == 0) {
      const int E = bad ? kBadExp : (c < 2 * m ? scale_exp(mx) : 0);
      sE[c] = E;
      xexp[(size_t)sh * kN + c] = E;
    }
  }
  __syncthreads();
  const int nj8 = npad / 8;
  for (int it = tid; it < kN * nj8; it += blockDim.x) {
    const int c = it / nj8, j8 = it % nj8;
    const int E = sE[c];
    unsigned short dg[8][kSl];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = j8 * 8 + e;
      double v = 0.0;
      if (c < 2 * m && j < n) {
        const cd x = Xh[j + (size_t)(c >> 1) * ldx];
        v = (c & 1) ? x.y : x.x;
      }
      digits8(v, E, dg[e]);
    }
    const int J = (j8 * 8) / kKS;
    const int off = tile_off(c, (j8 * 8) % kKS);
#pragma unroll
    for (int l = 0; l < kSl; ++l) {
      uint4 u;
      u.x = dg[0][l] | ((unsigned)dg[1][l] << 16);
      u.y = dg[2][l] | ((unsigned)dg[3][l] << 16);
      u.z = dg[4][l] | ((unsigned)dg[5][l] << 16);
      u.w = dg[6][l] | ((unsigned)dg[7][l] << 16);
      const size_t base = ((size_t)(sh * kSl + l) * KT + J) * kBT + off;
      Xs[base / 8] = u;
    }
  }
}

// issuer owning level t: whole levels, 9 products per issuer with four
// ({9, 2}, {8, 3}, {7, 4}, {6, 5}), 18 with two
__host__ __device__ constexpr int level_owner(int t) {
  return kIss == 1 ? 0 : kIss == 4 ? (t <= 5 ? t - 2 : 9 - t) : ((t <= 5 ? t - 2 : 9 - t) >= 2 ? 1 : 0);
}

// Work item = (row block I, active shift w), grouped 16 shifts at a time so
// that the CTAs resident together share H and Xhat tiles in L2.
constexpr int kGroup = 16;
__device__ __forceinline__ void task_coords(long long t, int RB, int cnt, int* I, int* w) {
  const long long full = (long long)(cnt / kGroup) * kGroup * RB;
  if (t < full) {
    const long long g = t / ((long long)kGroup * RB), r = t % ((long long)kGroup * RB);
    *I = (int)(r / kGroup);
    *w = (int)(g * kGroup + r % kGroup);
  } else {
    const int gl = cnt - (cnt / kGroup) * kGroup;
    const long long r = t - full;
    *I = (int)(r / gl);
    *w = (cnt / kGroup) * kGroup + (int)(r % gl);
  }
}

__global__ void __launch_bounds__(kM, kCtasPerSm) tc_residual_kernel(
    int n, int m, int npad, const uint4* __restrict__ Hs, const int* __restrict__ hexp,
    const uint4* __restrict__ Xs, const int* __restrict__ xexp, const double* __restrict__ R,
    const cd* __restrict__ shifts, const int* __restrict__ list, const int* __restrict__ count,
    const cd* __restrict__ X, long long ldx, float2* __restrict__ E, double* __restrict__ acc,
    int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  // two stage buffers, each: kSl H slice tiles (kAT) then kSl Xhat slice tiles (kBT)
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + kBuf * kStageBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kIss + kBuf);  // mbar[kIss + b]: loads of buffer b
  __shared__ double red[2][kM / 32];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int KT = npad / kKS, RB = npad / kM;
  const int cnt = *count;
  const uint32_t mb = smem_addr(mbar);
  const uint32_t sBase = smem_addr(smem);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kIss + kBuf; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb + 8u * q));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  uint32_t lphase[2] = {0u, 0u};
  bool pend[2] = {false, false};  // a bulk copy into buffer b not yet seen complete
  const uint32_t lmb = mb + 8u * kIss;
  bool failed = false;
  float ah[kN], al[kN];
  // copy the slice tiles of K stage J of (row block I, shift sh) into buffer b
  auto stage_in = [&](int I, int sh, int J, int b) {
    const uint32_t dst = sBase + (uint32_t)b * kStageBytes;
    if constexpr (kBulk) {
      // sixteen contiguous tiles: one thread, sixteen TMA bulk copies
      pend[b] = true;
      if (tid == 0) {
        const uint32_t lb = lmb + 8u * (uint32_t)b;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lb), "r"(kStageBytes)
                     : "memory");
        for (int k = 0; k < kSl; ++k)
          bulk_copy(dst + (uint32_t)(k * kAT * 2), Hs + ((size_t)(k * RB + I) * KT + J) * (kAT / 8),
                    (uint32_t)(kAT * 2), lb);
        for (int l = 0; l < kSl; ++l)
          bulk_copy(dst + (uint32_t)(kSl * kAT * 2 + l * kBT * 2),
                    Xs + ((size_t)(sh * kSl + l) * KT + J) * (kBT / 8), (uint32_t)(kBT * 2), lb);
      }
    } else {
      for (int v = tid; v < kSl * (kAT + kBT) / 8; v += kM) {
        const uint4* src;
        if (v < kSl * kAT / 8) {
          const int k = v / (kAT / 8), o = v % (kAT / 8);
          src = Hs + ((size_t)(k * RB + I) * KT + J) * (kAT / 8) + o;
        } else {
          const int vb = v - kSl * kAT / 8;
          const int l = vb / (kBT / 8), o = vb % (kBT / 8);
          src = Xs + ((size_t)(sh * kSl + l) * KT + J) * (kBT / 8) + o;
        }
        cp16(dst + (uint32_t)v * 16u, src);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  };
  // levels of one accumulation window (TMEM half `half`) into the double-float sums
  auto read_window = [&](uint32_t half) {
    float sc = 0.0078125f * 0.0078125f;  // 2^{-7t}, t = 2
#pragma unroll 1
    for (int lv = 0; lv < kLev; ++lv) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + half + (uint32_t)(lv * kN), r);
#pragma unroll
      for (int c = 0; c < kN; ++c) {
        const float p = __uint_as_float(r[c]) * sc;
        const float s = ah[c] + p;
        const float bp = s - ah[c];
        al[c] += (ah[c] - (s - bp)) + (p - bp);
        ah[c] = s;
      }
      sc *= 0.0078125f;
    }
  };
  for (long long t = blockIdx.x; t < (long long)cnt * RB && !failed; t += gridDim.x) {
    int I, w;
    task_coords(t, RB, cnt, &I, &w);
    const int sh = list[w];
    const int i0 = I * kM;
    const int J0 = max(0, i0 - m) / kKS;
    const int nst = KT - J0;
#pragma unroll
    for (int c = 0; c < kN; ++c) { ah[c] = 0.f; al[c] = 0.f; }
    if (kBuf == 2) stage_in(I, sh, J0, 0);
    for (int st = 0; st < nst; ++st) {
      const int b = kBuf == 2 ? (st & 1) : 0;
      if (kBuf == 1) stage_in(I, sh, J0 + st, 0);
      if constexpr (kBulk) {
        // the tiles land through the async proxy that the products read
        const bool lok = mbar_wait(lmb + 8u * (uint32_t)b, lphase[b]);
        if (__syncthreads_or(!lok)) {
          failed = true;
          break;
        }
        lphase[b] ^= 1u;
        pend[b] = false;
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
      }
      const uint32_t half = kTwoWin ? (uint32_t)(((st / kWin) & 1) * kLev * kN) : 0u;
      const int iss = tid >> 5;
      if ((tid & 31) == 0 && iss < kIss) {
        fence_after();
        const bool fresh = (st % kWin) == 0;
        const uint32_t aBase = sBase + (uint32_t)b * kStageBytes;
        const uint32_t bBase = aBase + (uint32_t)(kSl * kAT * 2);
        constexpr uint32_t kSbo = (uint32_t)kKG * 128u;
        // slice pair (k, l) into level t = k + l; the first product of each
        // level in a window overwrites, the rest accumulate
        auto issue = [&](int k, int l, int ks) {
          const int lv = k + l;
          const uint64_t ad = mat_desc(aBase + (uint32_t)((k - 1) * kAT * 2 + ks * 256), 128u, kSbo);
          const uint64_t bd = mat_desc(bBase + (uint32_t)((l - 1) * kBT * 2 + ks * 256), 128u, kSbo);
          const bool first = fresh && k == max(1, lv - kSl) && ks == 0;
          mma_bf16(tmem + half + (uint32_t)((lv - 2) * kN), ad, bd, kIdesc, first ? 0u : 1u);
        };
        static_assert(kIss == 1 || SSV_TC_INTERLEAVE == 0, "interleaving needs one issuer");
        if constexpr (SSV_TC_INTERLEAVE != 0) {
          // consecutive products go to different levels
#pragma unroll 1
          for (int ks = 0; ks < kKS / 16; ++ks)
#pragma unroll 1
            for (int k = 1; k <= kSl; ++k)
#pragma unroll 1
              for (int l = 1; l <= kSl + 1 - k; ++l) issue(k, l, ks);
        } else {
#pragma unroll 1
          for (int lv = 2; lv <= kSl + 1; ++lv) {
            if (level_owner(lv) != iss) continue;
#pragma unroll 1
            for (int k = max(1, lv - kSl); k <= min(kSl, lv - 1); ++k)
#pragma unroll
              for (int ks = 0; ks < kKS / 16; ++ks) issue(k, lv - k, ks);
          }
        }
        mma_commit(mb + 8u * (uint32_t)iss);
      }
      // the next stage streams into the other buffer (its MMAs completed
      // before the previous iteration ended) while these MMAs run
      if (kBuf == 2 && st + 1 < nst) stage_in(I, sh, J0 + st + 1, b ^ 1);
      // with two windows, the previous window's levels (the other TMEM half)
      // are read meanwhile
      if (kTwoWin && st > 0 && (st % kWin) == 0) {
        fence_after();
        read_window(half ^ (uint32_t)(kLev * kN));
        fence_before();
      }
      bool ok = true;
      for (int q = 0; q < kIss; ++q) ok = mbar_wait(mb + 8u * q, phase) && ok;
      phase ^= 1u;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      // with one window, it is read as soon as its last products are done
      if (!kTwoWin && ((st % kWin) == kWin - 1 || st == nst - 1)) {
        fence_after();
        read_window(0u);
        fence_before();
        __syncthreads();
      }
    }
    if (failed) break;
    if (kTwoWin) {
      fence_after();
      read_window((uint32_t)((((nst - 1) / kWin) & 1) * kLev * kN));
      fence_before();
    }
    // epilogue: E(i, q) = R(i, q) - (H Xhat)(i, q) + sigma Xhat(i, q)
    const int i = i0 + tid;
    double e2 = 0.0, x2 = 0.0;
    if (i < n) {
      const cd sigma = shifts[sh];
      const int Ei = hexp[i];
      const int* Ec = xexp + (size_t)sh * kN;
      const cd* Xh = X + (size_t)sh * m * ldx;
#pragma unroll
      for (int q = 0; q < kN / 2; ++q) {
        if (q < m) {
          const int er_ = Ec[2 * q], ei_ = Ec[2 * q + 1];
          const bool bad = Ei == kBadExp || er_ == kBadExp || ei_ == kBadExp;
          const double hxr = ldexp((double)ah[2 * q] + (double)al[2 * q], Ei + er_);
          const double hxi = ldexp((double)ah[2 * q + 1] + (double)al[2 * q + 1], Ei + ei_);
          const cd x = Xh[i + (size_t)q * ldx];
          double vr = -hxr + (sigma.x * x.x - sigma.y * x.y);
          double vi = -hxi + (sigma.x * x.y + sigma.y * x.x);
          if (i <= q) vr += R[i + (size_t)q * n];
          if (bad) vr = __longlong_as_double(0x7ff8000000000000LL);
          e2 += vr * vr + vi * vi;
          x2 += x.x * x.x + x.y * x.y;
          if (E != nullptr) E[(size_t)sh * n * m + i + (size_t)q * n] = make_float2((float)vr, (float)vi);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    }
    if ((tid & 31) == 0) {
      red[0][warp] = e2;
      red[1][warp] = x2;
    }
    __syncthreads();
    if (tid == 0) {
      double a = 0.0, bsum = 0.0;
      for (int k = 0; k < kM / 32; ++k) { a += red[0][k]; bsum += red[1][k]; }
      atomicAdd(acc + 2 * (size_t)sh, a);
      atomicAdd(acc + 2 * (size_t)sh + 1, bsum);
    }
    __syncthreads();
  }
  if (failed) {
    // a tensor-core completion never arrived: record it (every shift then
    // fails certification), give the MMAs in flight one more bounded wait,
    // drain this thread's copies, then release TMEM
    if (tid == 0) {
      atomicExch(err, 1);
      for (int q = 0; q < kIss; ++q) mbar_wait(mb + 8u * q, phase ^ 1u);
      if (kBulk)
        for (int b = 0; b < kBuf; ++b)
          if (pend[b]) mbar_wait(lmb + 8u * (uint32_t)b, lphase[b]);
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ---------------------------------------------------------------------------
// Two shifts per work item: the same digit products with N = 64 (the two
// shifts' Xhat slice tiles side by side form one 64-row B tile, since a 32-row
// tile is exactly four core-matrix row groups), so every H tile staged serves
// two shifts and each product is twice as large.  One CTA per SM (the eight
// levels x 64 columns fill TMEM), two stage buffers by TMA bulk copies, 256
// threads: thread (row, half) reads the 32 columns of one shift.
// ---------------------------------------------------------------------------
constexpr int kN2 = 64;
constexpr int kT2 = 2 * kM;
constexpr uint32_t kIdesc2 = idesc_bf16(kM, kN2);
constexpr uint32_t kStage2 = (uint32_t)kSl * (kAT + 2 * kBT) * 2;
constexpr size_t kSmem2 = 2 * (size_t)kStage2 + 128;
static_assert(kSmem2 <= 227 * 1024, "shared memory of the two-shift residual");
static_assert(kLev * kN2 <= 512, "TMEM columns of the two-shift residual");
constexpr int kWaitIss = SSV_TC_FUSED ? 1 : kIss;  // MMA barriers the two-shift kernel commits
constexpr int kPairGroup = 8;  // pairs that resident CTAs take together (L2 sharing of H tiles)

__device__ __forceinline__ void pair_coords(long long t, int RB, int np, int* I, int* w) {
  const long long full = (long long)(np / kPairGroup) * kPairGroup * RB;
  if (t < full) {
    const long long g = t / ((long long)kPairGroup * RB), r = t % ((long long)kPairGroup * RB);
    *I = (int)(r / kPairGroup);
    *w = (int)(g * kPairGroup + r % kPairGroup);
  } else {
    const int gl = np - (np / kPairGroup) * kPairGroup;
    const long long r = t - full;
    *I = (int)(r / gl);
    *w = (np / kPairGroup) * kPairGroup + (int)(r % gl);
  }
}

__global__ void __launch_bounds__(kT2, 1) tc_residual2_kernel(
    int n, int m, int npad, const uint4* __restrict__ Hs, const int* __restrict__ hexp,
    const uint4* __restrict__ Xs, const int* __restrict__ xexp, const double* __restrict__ R,
    const cd* __restrict__ shifts, const int* __restrict__ list, const int* __restrict__ count,
    const cd* __restrict__ X, long long ldx, float2* __restrict__ E, double* __restrict__ acc,
    int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + 2 * (size_t)kStage2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kIss + 2);  // mbar[kIss + b]: loads of buffer b
  __shared__ double red[2][kT2 / 32];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kM - 1), half = tid >> 7;
  const int KT = npad / kKS, RB = npad / kM;
  const int cnt = *count;
  const int npair = (cnt + 1) / 2;
  const uint32_t mb = smem_addr(mbar);
  const uint32_t lmb = mb + 8u * kIss;
  const uint32_t sBase = smem_addr(smem);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(kLev * kN2));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kIss + 2; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb + 8u * q));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  uint32_t lphase[2] = {0u, 0u};
  bool pend[2] = {false, false};
  bool failed = false;
  float ah[32], al[32];
  // K stage J of (row block I, shifts s0, s1 (s1 < 0: none)) into buffer b
  auto stage_in = [&](int I, int s0, int s1, int J, int b) {
    pend[b] = true;
    if (tid != 0) return;
    const uint32_t dst = sBase + (uint32_t)b * kStage2;
    const uint32_t lb = lmb + 8u * (uint32_t)b;
    const uint32_t bytes = (uint32_t)kSl * (kAT + (s1 >= 0 ? 2 : 1) * kBT) * 2;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lb), "r"(bytes) : "memory");
    for (int k = 0; k < kSl; ++k)
      bulk_copy(dst + (uint32_t)(k * kAT * 2), Hs + ((size_t)(k * RB + I) * KT + J) * (kAT / 8),
                (uint32_t)(kAT * 2), lb);
    for (int l = 0; l < kSl; ++l) {
      const uint32_t xb = dst + (uint32_t)(kSl * kAT * 2 + l * 2 * kBT * 2);
      bulk_copy(xb, Xs + ((size_t)(s0 * kSl + l) * KT + J) * (kBT / 8), (uint32_t)(kBT * 2), lb);
      if (s1 >= 0)
        bulk_copy(xb + (uint32_t)(kBT * 2), Xs + ((size_t)(s1 * kSl + l) * KT + J) * (kBT / 8),
                  (uint32_t)(kBT * 2), lb);
    }
  };
  // this thread's 32 columns of every level of one window into the double-float sums
  auto read_window = [&]() {
    float sc = 0.0078125f * 0.0078125f;  // 2^{-7t}, t = 2
#pragma unroll 1
    for (int lv = 0; lv < kLev; ++lv) {
      uint32_t r[32];
      tmem_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(lv * kN2 + half * 32), r);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float p = __uint_as_float(r[c]) * sc;
        const float s = ah[c] + p;
        const float bp = s - ah[c];
        al[c] += (ah[c] - (s - bp)) + (p - bp);
        ah[c] = s;
      }
      sc *= 0.0078125f;
    }
  };
  for (long long t = blockIdx.x; t < (long long)npair * RB && !failed; t += gridDim.x) {
    int I, w;
    pair_coords(t, RB, npair, &I, &w);
    const int s0 = list[2 * w];
    const int s1 = 2 * w + 1 < cnt ? list[2 * w + 1] : -1;
    const int i0 = I * kM;
    const int J0 = max(0, i0 - m) / kKS;
    const int nst = KT - J0;
#pragma unroll
    for (int c = 0; c < 32; ++c) { ah[c] = 0.f; al[c] = 0.f; }
    stage_in(I, s0, s1, J0, 0);
    for (int st = 0; st < nst; ++st) {
      const int b = st & 1;
      const bool lok = mbar_wait(lmb + 8u * (uint32_t)b, lphase[b]);
      if (__syncthreads_or(!lok)) {
        failed = true;
        break;
      }
      lphase[b] ^= 1u;
      pend[b] = false;
      const int iss = tid >> 5;
#if SSV_TC_FUSED
      // fused levels: the B digit tiles of a stage sit side by side (64 rows
      // each), so one product of H digit a against B digits b0 .. b0 + c - 1
      // (N = 64 c <= 256) lands digit b in TMEM level a + b; 24 products per
      // stage instead of 72.  The two products of a = 0 cover all eight
      // levels and open the window, so one thread issues everything in order.
      if (tid == 0) {
        fence_after();
        const bool fresh = (st % kWin) == 0;
        const uint32_t aBase = sBase + (uint32_t)b * kStage2;
        const uint32_t bBase = aBase + (uint32_t)(kSl * kAT * 2);
        constexpr uint32_t kSbo = (uint32_t)kKG * 128u;
#pragma unroll
        for (int ks = 0; ks < kKS / 16; ++ks) {
#pragma unroll
          for (int da = 0; da < kSl; ++da) {
#pragma unroll
            for (int b0 = 0; b0 < kSl - da; b0 += 4) {
              const int c = min(4, kSl - da - b0);
              const uint64_t ad = mat_desc(aBase + (uint32_t)(da * kAT * 2 + ks * 256), 128u, kSbo);
              const uint64_t bd = mat_desc(bBase + (uint32_t)(b0 * 2 * kBT * 2 + ks * 256), 128u, kSbo);
              const bool first = fresh && ks == 0 && da == 0;
              mma_bf16(tmem + (uint32_t)((da + b0) * kN2), ad, bd, idesc_bf16(kM, kN2 * c), first ? 0u : 1u);
            }
          }
        }
        mma_commit(mb);
      }
#else
      if ((tid & 31) == 0 && iss < kIss) {
        fence_after();
        const bool fresh = (st % kWin) == 0;
        const uint32_t aBase = sBase + (uint32_t)b * kStage2;
        const uint32_t bBase = aBase + (uint32_t)(kSl * kAT * 2);
        constexpr uint32_t kSbo = (uint32_t)kKG * 128u;
#pragma unroll 1
        for (int lv = 2; lv <= kSl + 1; ++lv) {
          if (level_owner(lv) != iss) continue;
#pragma unroll 1
          for (int k = max(1, lv - kSl); k <= min(kSl, lv - 1); ++k) {
#pragma unroll
            for (int ks = 0; ks < kKS / 16; ++ks) {
              const uint64_t ad = mat_desc(aBase + (uint32_t)((k - 1) * kAT * 2 + ks * 256), 128u, kSbo);
              const uint64_t bd =
                  mat_desc(bBase + (uint32_t)((lv - k - 1) * 2 * kBT * 2 + ks * 256), 128u, kSbo);
              const bool first = fresh && k == max(1, lv - kSl) && ks == 0;
              mma_bf16(tmem + (uint32_t)((lv - 2) * kN2), ad, bd, kIdesc2, first ? 0u : 1u);
            }
          }
        }
        mma_commit(mb + 8u * (uint32_t)iss);
      }
#endif
      (void)iss;
      // the next stage streams into the other buffer (its products finished
      // in the previous round)
      if (st + 1 < nst) stage_in(I, s0, s1, J0 + st + 1, b ^ 1);
      bool ok = true;
      for (int q = 0; q < kWaitIss; ++q) ok = mbar_wait(mb + 8u * q, phase) && ok;
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      phase ^= 1u;
      if ((st % kWin) == kWin - 1 || st == nst - 1) {
        fence_after();
        read_window();
        fence_before();
        __syncthreads();
      }
    }
    if (failed) break;
    // epilogue of this thread's shift: E(i, q) = R(i, q) - (H Xhat)(i, q) + sigma Xhat(i, q)
    const int sh = half == 0 ? s0 : s1;
    const int i = i0 + row;
    double e2 = 0.0, x2 = 0.0;
    if (sh >= 0 && i < n) {
      const cd sigma = shifts[sh];
      const int Ei = hexp[i];
      const int* Ec = xexp + (size_t)sh * kN;
      const cd* Xh = X + (size_t)sh * m * ldx;
#pragma unroll
      for (int q = 0; q < kN / 2; ++q) {
        if (q < m) {
          const int er_ = Ec[2 * q], ei_ = Ec[2 * q + 1];
          const bool bad = Ei == kBadExp || er_ == kBadExp || ei_ == kBadExp;
          const double hxr = ldexp((double)ah[2 * q] + (double)al[2 * q], Ei + er_);
          const double hxi = ldexp((double)ah[2 * q + 1] + (double)al[2 * q + 1], Ei + ei_);
          const cd x = Xh[i + (size_t)q * ldx];
          double vr = -hxr + (sigma.x * x.x - sigma.y * x.y);
          double vi = -hxi + (sigma.x * x.y + sigma.y * x.x);
          if (i <= q) vr += R[i + (size_t)q * n];
          if (bad) vr = __longlong_as_double(0x7ff8000000000000LL);
          e2 += vr * vr + vi * vi;
          x2 += x.x * x.x + x.y * x.y;
          if (E != nullptr) E[(size_t)sh * n * m + i + (size_t)q * n] = make_float2((float)vr, (float)vi);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, o);
      x2 += __shfl_xor_sync(0xffffffffu, x2, o);
    }
    if ((tid & 31) == 0) {
      red[0][warp] = e2;
      red[1][warp] = x2;
    }
    __syncthreads();
    if ((tid & (kM - 1)) == 0 && sh >= 0) {
      double a = 0.0, bsum = 0.0;
      for (int k = half * (kM / 32); k < (half + 1) * (kM / 32); ++k) { a += red[0][k]; bsum += red[1][k]; }
      atomicAdd(acc + 2 * (size_t)sh, a);
      atomicAdd(acc + 2 * (size_t)sh + 1, bsum);
    }
    __syncthreads();
  }
  if (failed) {
    // a completion never arrived: record it (every shift then fails
    // certification), give the products and copies in flight one more
    // bounded wait, then release TMEM
    if (tid == 0) {
      atomicExch(err, 1);
      for (int q = 0; q < kWaitIss; ++q) mbar_wait(mb + 8u * q, phase);
      for (int b = 0; b < 2; ++b)
        if (pend[b]) mbar_wait(lmb + 8u * (uint32_t)b, lphase[b]);
    }
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kLev * kN2));
}

__global__ void tc_identity_list_kernel(int s, int* __restrict__ list, int* __restrict__ count,
                                        double* __restrict__ acc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x) {
    list[i] = i;
    acc[2 * (size_t)i] = 0.0;
    acc[2 * (size_t)i + 1] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *count = s;
}

__global__ void tc_eta_kernel(int n, int m, int s, const double* __restrict__ hn,
                              const double* __restrict__ R, const cd* __restrict__ shifts,
                              const double* __restrict__ acc, const int* __restrict__ err,
                              double* __restrict__ eta) {
  const int sh = blockIdx.x * blockDim.x + threadIdx.x;
  if (sh >= s) return;
  double r2 = 0.0;
  for (int q = 0; q < m; ++q)
    for (int i = 0; i <= q && i < n; ++i) r2 = fma(R[i + (size_t)q * n], R[i + (size_t)q * n], r2);
  const cd sg = shifts[sh];
  const double m2 = fmax(hn[0] - 2.0 * sg.x * hn[1] + (double)n * (sg.x * sg.x + sg.y * sg.y), 0.0);
  const double den = sqrt(m2) * sqrt(acc[2 * (size_t)sh + 1]) + sqrt(r2);
  double e = den > 0.0 ? sqrt(acc[2 * (size_t)sh]) / den : (den == den ? 0.0 : den);
  if (*err != 0) e = __longlong_as_double(0x7ff8000000000000LL);
  eta[sh] = e;
}

}  // namespace

int resid_tc_npad(int n) { return (n + kM - 1) / kM * kM; }

int resid_tc_ktile() { return kKS; }

size_t resid_tc_hbytes(int n) {
  const size_t np = (size_t)resid_tc_npad(n);
  return ((size_t)kSl * np * np * 2 + 255) / 256 * 256 + (np * sizeof(int) + 255) / 256 * 256;
}

size_t resid_tc_xbytes(int n, int s) {
  const size_t np = (size_t)resid_tc_npad(n);
  return ((size_t)s * kSl * kN * np * 2 + 255) / 256 * 256 +
         ((size_t)s * kN * sizeof(int) + 255) / 256 * 256 + 256;
}

int resid_tc_split_h(const Handle* h, void* hbuf, cudaStream_t st) {
  const int n = h->n, m = h->m, np = resid_tc_npad(n);
  unsigned char* b = static_cast<unsigned char*>(hbuf);
  uint4* Hs = reinterpret_cast<uint4*>(b);
  int* hexp = reinterpret_cast<int*>(b + ((size_t)kSl * np * np * 2 + 255) / 256 * 256);
  tc_hrow_kernel<<<(np + 127) / 128, 128, 0, st>>>(n, m, np, h->H, hexp);
  count_launch();
  const long long items = (long long)np * (np / 8);
  const int grid = (int)std::min<long long>((items + 255) / 256, (long long)num_sms() * 16);
  tc_hsplit_kernel<<<grid, 256, 0, st>>>(n, m, np, h->H, hexp, Hs);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

int resid_tc_run(const Handle* h, const void* hbuf, void* xbuf, int s, const double* shifts,
                 const int* list, const int* count, const double* Xhat, long long ldx, void* E,
                 double* acc, int* err, cudaStream_t st) {
  const int n = h->n, m = h->m, np = resid_tc_npad(n);
  if (m > kN / 2) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  const unsigned char* hb = static_cast<const unsigned char*>(hbuf);
  const uint4* Hs = reinterpret_cast<const uint4*>(hb);
  const int* hexp = reinterpret_cast<const int*>(hb + ((size_t)kSl * np * np * 2 + 255) / 256 * 256);
  unsigned char* xb = static_cast<unsigned char*>(xbuf);
  uint4* Xs = reinterpret_cast<uint4*>(xb);
  int* xexp = reinterpret_cast<int*>(xb + ((size_t)s * kSl * kN * np * 2 + 255) / 256 * 256);
  const cd* X = reinterpret_cast<const cd*>(Xhat);
  tc_xsplit_kernel<<<s, 256, 0, st>>>(n, m, np, list, count, X, ldx, Xs, xexp);
  count_launch();
  if (kPairs) {
    SSV_CUDA_TRY(cudaFuncSetAttribute(tc_residual2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSmem2));
    const long long tasks = (long long)((s + 1) / 2) * (np / kM);
    const int grid = (int)std::max<long long>(1, std::min<long long>(tasks, (long long)num_sms()));
    tc_residual2_kernel<<<grid, kT2, kSmem2, st>>>(n, m, np, Hs, hexp, Xs, xexp, h->R,
                                                   reinterpret_cast<const cd*>(shifts), list, count, X,
                                                   ldx, static_cast<float2*>(E), acc, err);
  } else {
    SSV_CUDA_TRY(cudaFuncSetAttribute(tc_residual_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSmem));
    const long long tasks = (long long)s * (np / kM);
    const int grid =
        (int)std::max<long long>(1, std::min<long long>(tasks, (long long)num_sms() * kCtasPerSm));
    tc_residual_kernel<<<grid, kM, kSmem, st>>>(n, m, np, Hs, hexp, Xs, xexp, h->R,
                                                reinterpret_cast<const cd*>(shifts), list, count, X,
                                                ldx, static_cast<float2*>(E), acc, err);
  }
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

int backward_error_tc(const Handle* h, int s, const double* shifts, const double* Xhat,
                      long long ldx, double* eta, cudaStream_t st) {
  if (s == 0) return SSV_OK;
  if (h->m > kN / 2) return SSV_ENOTSUP;
  const size_t hb = resid_tc_hbytes(h->n), xb = resid_tc_xbytes(h->n, s);
  const size_t lb = ((size_t)s * sizeof(int) + 255) / 256 * 256;
  const size_t ab = ((size_t)2 * s * sizeof(double) + 255) / 256 * 256;
  unsigned char* buf = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&buf, hb + xb + lb + ab + 256, st));
  int* list = reinterpret_cast<int*>(buf + hb + xb);
  double* acc = reinterpret_cast<double*>(buf + hb + xb + lb);
  int* misc = reinterpret_cast<int*>(buf + hb + xb + lb + ab);  // count, err
  int rc = SSV_OK;
  cudaError_t e = cudaMemsetAsync(misc, 0, 2 * sizeof(int), st);
  if (e == cudaSuccess) {
    tc_identity_list_kernel<<<std::min(1024, (s + 255) / 256), 256, 0, st>>>(s, list, misc, acc);
    count_launch();
    rc = resid_tc_split_h(h, buf, st);
    if (rc == SSV_OK)
      rc = resid_tc_run(h, buf, buf + hb, s, shifts, list, misc, Xhat, ldx, nullptr, acc, misc + 1, st);
    if (rc == SSV_OK) {
      tc_eta_kernel<<<(s + 255) / 256, 256, 0, st>>>(h->n, h->m, s, h->hnorm2, h->R,
                                                    reinterpret_cast<const cd*>(shifts), acc,
                                                    misc + 1, eta);
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
