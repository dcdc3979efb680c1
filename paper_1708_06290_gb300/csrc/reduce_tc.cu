// Controller-Hessenberg reduction (Algorithm 1, Sec. 2) with two levels of
// blocking (Sec. 2.1: blocks of b columns, each split into mini-blocks of m
// columns; Algorithms 2 and 3, Eqs. for V, T and Y), where every product of
// O(n^3) total work runs on the tensor cores as an FP64-accurate product of
// error-free BF16 digits, and the panels stay in FP64.
//
// Arithmetic of the products.  An operand row (or column) is scaled by the
// power of two 2^E above its largest magnitude and cut into eight 7-bit
// digits (56 bits, more than FP64's 53).  The product of digit pair (a, b)
// over one K = 16 slice is a tcgen05.mma of kind::f16 into FP32 TMEM; pairs
// with a + b = t accumulate in level t.  The rank-b updates keep t = 0..7 (36 pairs; the
// dropped pairs weigh below 2^-53 of the product's scale, the row maximum
// times the column maximum); the long-K products A V_s and V^T A keep
// t = 0..8 (43 pairs, dropped part below 2^-60): their terms mostly sit far
// below that scale, and with eight levels their error grew to about ten
// times an FP64 product's.  One instruction serves several pairs: the B digit
// tiles of a stage sit side by side, so A digit a against B digits b0 .. b0+c-1
// (N c <= 256 columns) lands digit b in level a + b (fused levels).  A level's
// sums are integers below 2^24 for K <= 128 (8 pairs x 128 x 127^2 < 2^24),
// hence exact in FP32; after each window of 128 the levels are added exactly into 64-bit
// fixed-point words (levels 0-3, 4-7 and 8; a window adds below 2^46 to a
// word), kept across the whole K range and turned into FP64 once per output.
//
// A column of the V factor of a block's reflectors has entries of magnitude
// <= 1 with a unit pivot (|v_r| <= 1 because |alpha - beta| >= |beta| >=
// |x_r|), so V by columns uses the fixed exponent 1 and the panel kernel
// writes those digits as the reflectors appear; V by rows (mostly far below
// 1) is split with per-row exponents at the end of the block.
//
// Per block of jb reflectors (rows r0 = z + m .. n-1, trailing columns
// z + b ..):
//   per mini-block (panel kernel, cooperative, FP64):
//     P <- P - Y V(cols, :)^T  (from the right),  P <- P - V T^T V^T P  (left),
//     Householder QR of the mini-block, T's new columns (Eq. for T),
//   then Y's new columns (Eq. for Y): Y_s = (A V_s - Y V^T V_s) T_s, with
//     A V_s on the tensor cores (A = the matrix at the start of the block);
//   block end (Algorithm 3, all on the tensor cores but the T^T product):
//     A(:, z+m:) -= Y V^T  (rows above r0 and C: from column z + m; rows r0..:
//                           from column z + b),
//     W = V^T A(r0:, z+b:),  Z = T^T W,  A(r0:, z+b:) -= V Z.
// Step 1 of Algorithm 1 (the QR of B, applied to A from both sides and to C
// from the right) is one more block with r0 = 0 and no block columns.
//
// The working matrix E stacks C (rows 0..p-1) above A (rows p..p+n-1),
// column-major, so that every right update of A and C is one product.
//
// Every wait (grid barrier, mbarrier) is bounded and raises an error flag;
// the host then reports SSV_ETIMEOUT.
#include <algorithm>
#include <climits>

#include "tc_common.cuh"

namespace ssv {

namespace {

using namespace tcg;

constexpr int kTR = 64;                  // rows of a digit tile
constexpr int kTK = 32;                  // K of a digit tile
constexpr int kTileEl = kTR * kTK;       // 2048 BF16 values (4 KB) in the core-matrix layout
constexpr int kD = kDigits;              // digits per operand value
constexpr int kBmax = 128;               // reflectors per block at most
constexpr int kMaxW = 64;                // mini-block width (m) at most
constexpr int kWinTiles = 4;             // K tiles per exact window (4 x 32 = 128)
constexpr int kGT = 256;                 // threads of the product kernel
constexpr int kIssuers = 1;              // MMA completion barriers (one issuing thread)
constexpr unsigned long long kSpin = 1ull << 26;  // grid barrier naps before giving up

// Debug builds (-DSSV_BOUNDS_CHECK): every global index of these kernels is
// checked against its buffer's extent; one out of range is clamped to 0 (a
// bulk copy then stays inside its buffer) and sets bit 2 of the error word,
// so the reduction fails.  The scratch is filled with NaN before use and a
// canary after it is verified at the end.  In normal builds RBCK(i, n, e) is i.
#ifdef SSV_BOUNDS_CHECK
__device__ __forceinline__ size_t rbck(long long i, size_t n, int* err) {
  if (i < 0 || (size_t)i >= n) {
    if (err) atomicOr(err, 2);
    return 0;
  }
  return (size_t)i;
}
// [i, i + len) inside [0, n)
__device__ __forceinline__ size_t rbcr(long long i, long long len, size_t n, int* err) {
  if (i < 0 || (size_t)(i + len) > n) {
    if (err) atomicOr(err, 2);
    return 0;
  }
  return (size_t)i;
}
#define RBCK(i, n, e) rbck((long long)(i), (size_t)(n), (e))
#define RBCR(i, len, n, e) rbcr((long long)(i), (long long)(len), (size_t)(n), (e))
#else
#define RBCK(i, n, e) ((size_t)(i))
#define RBCR(i, len, n, e) ((size_t)(i))
#endif

// Digit tiles of an R x K operand (R rows, each scaled by 2^ex[r]): tile
// (digit, J, I) holds rows 64 I .. 64 I + 63 and K 32 J .. 32 J + 31, the
// tiles of one (digit, J) consecutive in I, so that two neighbours are the
// 128-row A operand of one product.
struct DigitMat {
  unsigned short* d;
  int* ex;    // per row; null: the fixed exponent 1
  int RT;     // 64-row tiles (even)
  int KT;     // 32-wide K tiles
  size_t nd;  // BF16 values in d (the extent the debug build checks)
};

__host__ __device__ __forceinline__ size_t tile_index(const DigitMat& M, int dig, int J, int I) {
  return (((size_t)dig * M.KT + J) * M.RT + I) * kTileEl;
}

// bit pattern of the BF16 digit `l` of x at exponent E
__device__ __forceinline__ void digits_of(double x, int E, unsigned short (&d)[kD]) { digits8(x, E, d); }

// ---------------------------------------------------------------------------
// Splitting.  Element (r, k) of the source is src[r * sr + k * sk]; rows
// [r_lo, r_hi) and K [k_lo, k_hi) are taken, everything else of a tile is 0.
// ---------------------------------------------------------------------------

// exponent pass: ex[r] = max over the K range of scale_exp(|x|) (ex preset to INT_MIN)
__global__ void __launch_bounds__(256) split_exp_kernel(const double* __restrict__ src, long long sr,
                                                        long long sk, int r_lo, int r_hi, int k_lo,
                                                        int k_hi, int kchunk, int* __restrict__ ex,
                                                        size_t nsrc, size_t nex, int* err) {
  const int tid = threadIdx.x;
  const int rb = r_lo + blockIdx.x * 64;
  const int kb = k_lo + blockIdx.y * kchunk;
  const int ke = min(k_hi, kb + kchunk);
  if (sk == 1) {
    // K contiguous: a warp per row, lanes along K
    const int lane = tid & 31, wp = tid >> 5;
    for (int rr = wp; rr < 64; rr += 8) {
      const int r = rb + rr;
      if (r >= r_hi) break;
      double mx = 0.0;
      for (int k = kb + lane; k < ke; k += 32) mx = fmax(mx, fabs(src[RBCK((size_t)r * sr + k, nsrc, err)]));
      for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) atomicMax(ex + RBCK(r, nex, err), scale_exp(mx));
    }
  } else {
    // rows contiguous (sr == 1 in every use): threads along rows, four K groups
    __shared__ double part[4][64];
    const int rr = tid & 63, g = tid >> 6;
    const int r = rb + rr;
    double mx = 0.0;
    if (r < r_hi)
      for (int k = kb + g; k < ke; k += 4)
        mx = fmax(mx, fabs(src[RBCK((size_t)r * sr + (size_t)k * sk, nsrc, err)]));
    part[g][rr] = mx;
    __syncthreads();
    if (g == 0 && r < r_hi) {
      mx = fmax(fmax(part[0][rr], part[1][rr]), fmax(part[2][rr], part[3][rr]));
      atomicMax(ex + RBCK(r, nex, err), scale_exp(mx));
    }
  }
}

// digit pass: one CTA per tile (I, J) of [I0, I0 + gridDim.x) x [J0, J0 + gridDim.y)
__global__ void __launch_bounds__(256) split_dig_kernel(const double* __restrict__ src, long long sr,
                                                        long long sk, int r_lo, int r_hi, int k_lo,
                                                        int k_hi, DigitMat M, int I0, int J0, size_t nsrc,
                                                        size_t nex, int* err) {
  __shared__ double t[kTR][kTK + 1];
  const int tid = threadIdx.x;
  const int I = I0 + blockIdx.x, J = J0 + blockIdx.y;
  const int rb = I * kTR, kb = J * kTK;
  for (int e = tid; e < kTileEl; e += 256) {
    int rr, kk;
    if (sk == 1) { rr = e / kTK; kk = e % kTK; }
    else { rr = e % kTR; kk = e / kTR; }
    const int r = rb + rr, k = kb + kk;
    double v = 0.0;
    if (r >= r_lo && r < r_hi && k >= k_lo && k < k_hi) v = src[RBCK((size_t)r * sr + (size_t)k * sk, nsrc, err)];
    t[rr][kk] = v;
  }
  __syncthreads();
  const int rr = tid >> 2, kq = (tid & 3) * 8;
  const int r = rb + rr;
  int E = (r >= r_lo && r < r_hi) ? (M.ex ? M.ex[RBCK(r, nex, err)] : 1) : 0;
  if (E < -4000) E = 0;  // a row with an empty K range (all of its values are 0)
  unsigned short dg[8][kD];
#pragma unroll
  for (int q = 0; q < 8; ++q) digits_of(t[rr][kq + q], E, dg[q]);
  const size_t off = (size_t)tile_off_kg(rr, kq, kTK / 8);
#pragma unroll
  for (int l = 0; l < kD; ++l) {
    uint4 v;
    v.x = (unsigned)dg[0][l] | ((unsigned)dg[1][l] << 16);
    v.y = (unsigned)dg[2][l] | ((unsigned)dg[3][l] << 16);
    v.z = (unsigned)dg[4][l] | ((unsigned)dg[5][l] << 16);
    v.w = (unsigned)dg[6][l] | ((unsigned)dg[7][l] << 16);
    *reinterpret_cast<uint4*>(M.d + RBCR(tile_index(M, l, J, I) + off, 8, M.nd, err)) = v;
  }
}


// ---------------------------------------------------------------------------
// The digit product: output (r + roff, c + coff) for A rows r in [M0, M1)
// and B rows c in [N0, N1) (column-major C, leading dimension ldc) receives
// x = sum_k A(r, k) B(c, k), k over the K tiles [J0, J1).  sub: C -= x, else
// C = x; with ksplit > 1 chunk s of the K range writes C + s * kstride.
// ---------------------------------------------------------------------------
struct GSeg {
  DigitMat A, B;
  int J0, J1;
};
struct GArgs {
  GSeg seg;
  int M0, M1, N0, N1;
  int roff, coff;
  double* C;
  size_t nc;  // doubles from C on (the extent the debug build checks)
  long long ldc;
  int sub;
  int ksplit;
  long long kstride;
  int* err;
};

template <int NT, int LV>
struct GCfg {
  static constexpr uint32_t kABytes = 2u * kTileEl * 2u;        // 128 rows x 32 K of one digit
  static constexpr uint32_t kBBytes = (uint32_t)NT * kTK * 2u;  // NT rows x 32 K of one digit
  // A digit planes, B digit planes, then one B plane of zeros (written once)
  // so that the first fused product of a window covers every level
  static constexpr uint32_t kStage = (uint32_t)kD * (kABytes + kBBytes) + kBBytes;
  // stage buffers: three when they fit (N = 16: two loads in flight), else two
  static constexpr int kNS = 3 * (size_t)kStage + 256 <= 227 * 1024 ? 3 : 2;
  static constexpr size_t kSmem = kNS * (size_t)kStage + 256;
  static constexpr uint32_t kUsed = (uint32_t)LV * NT;
  static constexpr uint32_t kCols = kUsed <= 32 ? 32 : kUsed <= 64 ? 64 : kUsed <= 128 ? 128 : kUsed <= 256 ? 256 : 512;
  static_assert(kSmem <= 227 * 1024, "shared memory of the digit product");
  static_assert(kUsed <= 512, "TMEM columns");
  static_assert(LV == 8 || LV == 9, "levels");
};

template <int CPT>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[CPT]) {
  if constexpr (CPT == 8) tmem_ld8(taddr, r);
  else if constexpr (CPT == 16) tmem_ld16(taddr, r);
  else tmem_ld32(taddr, r);
}

// 2^e as a double (e may leave the normal range only for absurd inputs)
__device__ __forceinline__ double pow2(int e) {
  if (e > -1022 && e < 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}

template <int NT, int LV>
__global__ void __launch_bounds__(kGT, 1) tc_gemm_kernel(GArgs g) {
  using Cfg = GCfg<NT, LV>;
  constexpr int CPT = NT / 2;
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int NS = Cfg::kNS;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(smem + NS * (size_t)Cfg::kStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + kIssuers + NS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, half = warp >> 2;
  const uint32_t mb = smem_addr(mbar);
  const uint32_t lmb = mb + 8u * kIssuers;  // lmb + 8 b: loads of stage buffer b
  const uint32_t sBase = smem_addr(smem);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                 "r"(Cfg::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kIssuers + NS; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb + 8u * q));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int bq = 0; bq < NS; ++bq) {
    uint4* zp = reinterpret_cast<uint4*>(smem + (size_t)bq * Cfg::kStage + kD * (Cfg::kABytes + Cfg::kBBytes));
    for (int e = tid; e < (int)(Cfg::kBBytes / 16); e += kGT) zp[e] = make_uint4(0u, 0u, 0u, 0u);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the zeros, seen by the tensor cores
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;
  uint32_t phase = 0;
  uint32_t lphase[3] = {0u, 0u, 0u};
  bool pend[3] = {false, false, false};
  bool failed = false;
  const int iI0 = g.M0 / 128, iI1 = (g.M1 + 127) / 128;
  const int iN0 = g.N0 / NT, iN1 = (g.N1 + NT - 1) / NT;
  const int nI = max(0, iI1 - iI0), nN = max(0, iN1 - iN0);
  const long long ntile = (long long)nI * nN * g.ksplit;
  const DigitMat& A = g.seg.A;
  const DigitMat& B = g.seg.B;
  constexpr int NW = (LV + 3) / 4;  // 64-bit words of the level sums
  struct Tile {
    int iI, n0, ks, jlo, nst;
  };
  auto tile_of = [&](long long tt) {
    Tile t;
    t.n0 = (iN0 + (int)(tt % nN)) * NT;
    t.iI = iI0 + (int)((tt / nN) % nI);
    t.ks = (int)(tt / ((long long)nN * nI));
    int jlo = g.seg.J0, jhi = g.seg.J1;
    if (g.ksplit > 1) {
      int chunk = (jhi - jlo + g.ksplit - 1) / g.ksplit;
      chunk = (chunk + kWinTiles - 1) / kWinTiles * kWinTiles;
      jlo = jlo + t.ks * chunk;
      jhi = min(jhi, jlo + chunk);
    }
    t.jlo = jlo;
    t.nst = max(0, jhi - jlo);
    return t;
  };
  // stage st of tile t into buffer b
  auto stage_in = [&](const Tile& t, int st, int b) {
    pend[b] = true;
    if (tid != 0) return;
    const int J = t.jlo + st;
    const uint32_t dst = sBase + (uint32_t)b * Cfg::kStage;
    const uint32_t lb = lmb + 8u * (uint32_t)b;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(lb),
                 "r"(Cfg::kStage - Cfg::kBBytes)
                 : "memory");
    for (int d = 0; d < kD; ++d)
      bulk_copy(dst + (uint32_t)d * Cfg::kABytes,
                A.d + RBCR(tile_index(A, d, J, 2 * t.iI), 2 * kTileEl, A.nd, g.err), Cfg::kABytes, lb);
    for (int d = 0; d < kD; ++d)
      bulk_copy(dst + kD * Cfg::kABytes + (uint32_t)d * Cfg::kBBytes,
                B.d + RBCR(tile_index(B, d, J, t.n0 / kTR) + (size_t)(t.n0 % kTR) * kTK, NT * kTK, B.nd, g.err),
                Cfg::kBBytes, lb);
  };
  bool prefetched = false;  // the first stages of this CTA's next tile are already in flight
  for (long long tt = blockIdx.x; tt < ntile && !failed; tt += gridDim.x) {
    const Tile cur = tile_of(tt);
    const int i0 = cur.iI * 128, n0 = cur.n0, ks = cur.ks;
    const int nst = cur.nst;
    // exact level sums of every window, in 64-bit words: word w holds levels
    // 4w .. 4w + 3, level L at bit 21 - 7 (L - 4 w); a window adds less than
    // 2^46 to a word, so 2^17 windows (K up to 16 M) cannot overflow it
    long long wacc[NW][CPT];
#pragma unroll
    for (int w = 0; w < NW; ++w)
#pragma unroll
      for (int c = 0; c < CPT; ++c) wacc[w][c] = 0;
    if (!prefetched)
      for (int q = 0; q < NS - 1 && q < nst; ++q) stage_in(cur, q, q);
    prefetched = false;
    for (int st = 0; st < nst; ++st) {
      const int b = st % NS;
      const bool lok = mbar_wait(lmb + 8u * (uint32_t)b, lphase[b]);
      if (__syncthreads_or(!lok)) {
        failed = true;
        break;
      }
      lphase[b] ^= 1u;
      pend[b] = false;
      if (tid == 0) {
        // fused levels: the B digit planes of a stage sit side by side (NT rows
        // each, then the zero plane), so one product of A digit a against B
        // digits b0 .. b0 + c - 1 (N = NT c <= 256) lands digit b in TMEM level
        // a + b; the products of a = 0 reach every level (the zero plane stands
        // for B digit 8) and open the window, so one thread issues them all
        fence_after();
        const bool fresh = (st % kWinTiles) == 0;
        const uint32_t aBase = sBase + (uint32_t)b * Cfg::kStage;
        const uint32_t bBase = aBase + kD * Cfg::kABytes;
        constexpr int kMaxC = 256 / NT;
#pragma unroll
        for (int kk = 0; kk < kTK / 16; ++kk) {
#pragma unroll
          for (int a = 0; a < kD; ++a) {
            const int nb = a == 0 ? LV : LV - a;  // B digits 0 .. nb - 1 (digit 8: the zero plane)
#pragma unroll
            for (int b0 = 0; b0 < nb; b0 += kMaxC) {
              const int c = min(kMaxC, nb - b0);
              const uint64_t ad = mat_desc(aBase + (uint32_t)a * Cfg::kABytes + (uint32_t)kk * 256u, 128u, 512u);
              const uint64_t bd = mat_desc(bBase + (uint32_t)b0 * Cfg::kBBytes + (uint32_t)kk * 256u, 128u, 512u);
              mma_bf16(tmem + (uint32_t)((a + b0) * NT), ad, bd, idesc_bf16(128, NT * c),
                       (fresh && kk == 0 && a == 0) ? 0u : 1u);
            }
          }
        }
        mma_commit(mb);
      }
      // the buffer of stage st - 1 (its products finished last round) takes stage st + NS - 1
      if (st + NS - 1 < nst) stage_in(cur, st + NS - 1, (st + NS - 1) % NS);
      const bool ok = mbar_wait(mb, phase);
      if (__syncthreads_or(!ok)) {
        failed = true;
        break;
      }
      phase ^= 1u;
      if (st == nst - 1 && tt + gridDim.x < ntile) {
        // every buffer is free: the next tile's first stages stream in during
        // the drain and the epilogue of this one
        const Tile nx = tile_of(tt + gridDim.x);
        for (int q = 0; q < NS - 1 && q < nx.nst; ++q) stage_in(nx, q, q);
        prefetched = true;
      }
      if ((st % kWinTiles) == kWinTiles - 1 || st == nst - 1) {
        fence_after();
#pragma unroll
        for (int w = 0; w < NW; ++w) {
#pragma unroll 1
          for (int L = 4 * w; L < min(LV, 4 * w + 4); ++L) {
            uint32_t rv[CPT];
            tmem_ld_cols<CPT>(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(L * NT + half * CPT), rv);
            const int sh = 21 - 7 * (L - 4 * w);
#pragma unroll
            for (int c = 0; c < CPT; ++c) wacc[w][c] += (long long)__float2int_rn(__uint_as_float(rv[c])) << sh;
          }
        }
        fence_before();
        __syncthreads();
      }
    }
    if (failed) break;
    // epilogue: word w weighs 2^{Ea + Eb - 35 - 28 w}; all loads of C first
    const int r = i0 + quarter * 32 + lane;
    if (r >= g.M0 && r < g.M1) {
      const int Ea = A.ex ? A.ex[RBCK(r, (size_t)A.RT * kTR, g.err)] : 1;
      const size_t c0 = (size_t)ks * g.kstride + (size_t)(r + g.roff);  // C offset of column 0
      double x[CPT];
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        const int col = n0 + half * CPT + c;
        const int Eb = (col >= g.N0 && col < g.N1) ? (B.ex ? B.ex[RBCK(col, (size_t)B.RT * kTR, g.err)] : 1) : 0;
        double v = 0.0;
        if (Ea == kBadExp || Eb == kBadExp) {
          v = __longlong_as_double(0x7ff8000000000000LL);
        } else if (Ea > -4000 && Eb > -4000) {
#pragma unroll
          for (int w = NW - 1; w >= 0; --w) v = fma((double)wacc[w][c], pow2(Ea + Eb - 35 - 28 * w), v);
        }
        x[c] = v;
      }
      auto cidx = [&](int col) { return RBCK(c0 + (long long)(col + g.coff) * g.ldc, g.nc, g.err); };
      if (g.sub) {
        double old[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int col = n0 + half * CPT + c;
          old[c] = (col >= g.N0 && col < g.N1) ? g.C[cidx(col)] : 0.0;
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int col = n0 + half * CPT + c;
          if (col >= g.N0 && col < g.N1) g.C[cidx(col)] = old[c] - x[c];
        }
      } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
          const int col = n0 + half * CPT + c;
          if (col >= g.N0 && col < g.N1) g.C[cidx(col)] = x[c];
        }
      }
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicExch(g.err, 1);
      mbar_wait(mb, phase);
      for (int b = 0; b < NS; ++b)
        if (pend[b]) mbar_wait(lmb + 8u * (uint32_t)b, lphase[b]);
    }
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols));
}

// ---------------------------------------------------------------------------
// Panel of one mini-block (Algorithm 2 between two updates of Y), one
// cooperative launch: CTA g owns a contiguous range of the panel rows
// r0 .. n-1, kept in shared memory (column-major per CTA); cross-CTA sums go
// through per-CTA partial slots and a bounded grid barrier.
// ---------------------------------------------------------------------------
constexpr int kPT = 256;
constexpr int kPartW = 8192;             // partial-sum slot per CTA (doubles)
constexpr int kPanRowsW = 8192;          // rows x columns of the panel per CTA at most
constexpr int kRedW = 0;                 // W = V^T P (j x w)
constexpr int kRedZ = 4096;              // Z = T^T W
constexpr int kRedPiv = 8192;            // pivot rows of the QR (two slots of 64)
constexpr int kRedS = 8192 + 128;        // S = V^T V_s ((j + wp) x wp)
constexpr int kRedTotal = kRedS + 8192;
constexpr size_t kPanFixed = 4096 + 4096 + 256 + 64 * 3 + 8 + 8 * kBmax;  // doubles besides the panel

struct PanArgs {
  double* P;          // panel column t, matrix row r: P[r + t * ldp]
  long long ldp;
  int r0, n;          // panel rows [r0, n)
  int w, wp;          // panel columns; reflectors generated (wp <= w)
  int pv0;            // pivot row of reflector t: pv0 + t
  int j;              // reflectors of the block before this mini-block
  int c0;             // matrix column of panel column 0 (rows c0.. of V: the right update)
  double* V;          // V(r, i) = V[r + i * ldv], explicit zeros and unit pivots
  long long ldv;
  double* T;          // T(i, k) = T[i + k * kBmax], upper triangular
  const double* Y;    // Y(matrix row r, i) = Y[yoff + r + i * ldy]
  long long ldy;
  int yoff;
  double* tau;        // tau of reflector t at tau[t]
  DigitMat vcol;      // V's digits, operand row = reflector, K = r (exponent 1: the unit pivot is
                      // every reflector's largest entry)
  double* part;       // [3][G][kPartW]
  double* red;        // kRedTotal
  unsigned* bar;      // this launch's arrival counter (zero at its start)
  int* err;
  // extents (doubles from each pointer on) the debug build checks
  size_t np, nv, ny, ntau, npart;
};

// Grid-wide barrier with a bounded wait: false once any CTA has given up.
// *bar counts this launch's arrivals (every panel launch has a counter of its
// own, zeroed at the start of the reduction); the k-th barrier completes when
// it reaches k * gridDim.x, so a CTA waits for the multiple of gridDim.x at or
// above its own arrival.
__device__ bool grid_sync(unsigned* bar, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    const unsigned target = (arrived + gridDim.x - 1) / gridDim.x * gridDim.x;
    unsigned long long spins = 0;
    for (;;) {
      unsigned now;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(now) : "l"(bar) : "memory");
      if ((int)(now - target) >= 0) break;
      if (*(volatile int*)err != 0) break;
      if (++spins > kSpin) {
        atomicExch(err, 1);
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
    __threadfence();
    s_ok = (*(volatile int*)err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}

// Sums with every thread of the CTA: out(e) = sum_k term(e, k) for e in
// [e0, e1), k < count(e); tpe threads (a power of two <= 32, the largest with
// tpe (e1 - e0) <= kPT) share an output, each taking every tpe-th k eight at
// a time, then a shuffle tree.  The order is fixed, so every CTA that forms the
// same sums gets the same bits.
template <typename Count, typename Term, typename Store>
__device__ __forceinline__ void block_sums(int e0, int e1, Count count, Term term, Store store) {
  const int nE = e1 - e0;
  if (nE <= 0) return;
  int tpe = 32;
  while (tpe > 1 && tpe * nE > kPT) tpe >>= 1;
  const int per = kPT / tpe;
  const int t = threadIdx.x, sub = t % tpe;
  for (int c0 = 0; c0 < nE; c0 += per) {
    const int el = c0 + t / tpe;
    const bool act = el < nE;
    const int e = e0 + el;
    double acc = 0.0;
    if (act) {
      const int K = count(e);
      int k = sub;
      for (; k + 7 * tpe < K; k += 8 * tpe) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = term(e, k + q * tpe);
        acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
      }
      for (; k < K; k += tpe) acc += term(e, k);
    }
    for (int o = tpe >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (act && sub == 0) store(e, acc);
  }
}

__device__ __forceinline__ void put_digits_v(const DigitMat& M, int row, int k, double v, int* err) {
  unsigned short d[kD];
  digits_of(v, 1, d);
  const size_t off = (size_t)tile_off_kg(row % kTR, k % kTK, kTK / 8);
#pragma unroll
  for (int l = 0; l < kD; ++l) M.d[RBCK(tile_index(M, l, k / kTK, row / kTR) + off, M.nd, err)] = d[l];
  (void)err;
}

__global__ void __launch_bounds__(kPT, 1) panel_kernel(PanArgs a) {
  extern __shared__ double psm[];
  const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int w = a.w, wp = a.wp, j = a.j;
  const int L = a.n - a.r0;
  const int rpc = (L + G - 1) / G;
  const int ra = a.r0 + g * rpc;
  const int nr = max(0, min(a.n, ra + rpc) - ra);
  double* Ps = psm;                      // Ps[t * rpc + rl]
  double* Vc = Ps + (size_t)rpc * w;     // Vc[t * j + i] = V(c0 + t, i)
  double* Zs = Vc + 4096;                // Zs[i * w + t]
  double* rs = Zs + 4096;                // 4 x 64 block partials
  double* dots = rs + 256;
  double* piv = dots + 64;
  double* taus = piv + 64;
  double* misc = taus + 64;
  double* tw = misc + 8;                 // 8 warps x kBmax: a row of T
  auto slot = [&](int q, int gg) { return a.part + RBCR(((size_t)q * G + gg) * kPartW, kPartW, a.npart, a.err); };
  // checked element accesses (plain indexing in normal builds)
  auto Pi = [&](long long i) -> double& { return a.P[RBCK(i, a.np, a.err)]; };
  auto Vi = [&](long long i) -> double& { return a.V[RBCK(i, a.nv, a.err)]; };
  auto Ti = [&](long long i) -> double& { return a.T[RBCK(i, (size_t)kBmax * kBmax, a.err)]; };
  auto Ri = [&](long long i) { return a.red + RBCK(i, (size_t)kRedTotal, a.err); };
  // partial e of CTA gg in slot q
  auto Pt = [&](int q, int gg, int e) { return a.part + RBCK(((size_t)q * G + gg) * kPartW + e, a.npart, a.err); };

  for (int e = tid; e < nr * w; e += kPT) {
    const int rl = e % nr, t = e / nr;
    Ps[t * rpc + rl] = Pi((size_t)(ra + rl) + (size_t)t * a.ldp);
  }
  if (j > 0) {
    // from the right: P -= Y(rows, 0:j) V(c0:c0+w, 0:j)^T
    for (int e = tid; e < w * j; e += kPT) {
      const int t = e % w, i = e / w;
      Vc[t * j + i] = Vi((size_t)(a.c0 + t) + (size_t)i * a.ldv);
    }
    __syncthreads();
    for (int e = tid; e < nr * w; e += kPT) {
      const int rl = e % nr, t = e / nr;
      const size_t y0 = (size_t)a.yoff + ra + rl;
      double acc = Ps[t * rpc + rl];
      for (int i = 0; i < j; ++i) acc = fma(-a.Y[RBCK(y0 + (size_t)i * a.ldy, a.ny, a.err)], Vc[t * j + i], acc);
      Ps[t * rpc + rl] = acc;
    }
    __syncthreads();
    // from the left: W = V^T P, Z = T^T W, P -= V Z
    double* my = slot(0, g);
    for (int e = tid; e < j * w; e += kPT) {
      const int i = e / w, t = e % w;
      const size_t v0 = (size_t)ra + (size_t)i * a.ldv;
      double acc = 0.0;
      for (int rl = 0; rl < nr; ++rl) acc = fma(Vi(v0 + rl), Ps[t * rpc + rl], acc);
      my[RBCK(e, kPartW, a.err)] = acc;
    }
    if (!grid_sync(a.bar, a.err)) return;
    const int ch = (j * w + G - 1) / G;
    const int e0 = min(j * w, g * ch), e1 = min(j * w, (g + 1) * ch);
    block_sums(
        e0, e1, [&](int) { return G; }, [&](int e, int gg) { return __ldcg(Pt(0, gg, e)); },
        [&](int e, double v) { *Ri(kRedW + e) = v; });
    if (!grid_sync(a.bar, a.err)) return;
    block_sums(
        e0, e1, [&](int e) { return e / w + 1; },
        [&](int e, int k) { return Ti(k + (size_t)(e / w) * kBmax) * __ldcg(Ri(kRedW + k * w + e % w)); },
        [&](int e, double v) { *Ri(kRedZ + e) = v; });
    if (!grid_sync(a.bar, a.err)) return;
    for (int e = tid; e < j * w; e += kPT) Zs[e] = __ldcg(Ri(kRedZ + e));
    __syncthreads();
    for (int e = tid; e < nr * w; e += kPT) {
      const int rl = e % nr, t = e / nr;
      const size_t v0 = (size_t)ra + rl;
      double acc = Ps[t * rpc + rl];
      for (int i = 0; i < j; ++i) acc = fma(-Vi(v0 + (size_t)i * a.ldv), Zs[i * w + t], acc);
      Ps[t * rpc + rl] = acc;
    }
  }
  __syncthreads();
  // Householder QR of the mini-block: reflector t zeroes rows > pv0 + t of column t
  for (int t = 0; t < wp; ++t) {
    const int pr = a.pv0 + t;
    const int nk = w - t;  // columns t .. w-1 (k = t: the squared norm below the pivot)
    {
      const int kk = tid & 63, grp = tid >> 6;
      double acc = 0.0;
      if (kk < nk) {
        const double* ck = Ps + (size_t)(t + kk) * rpc;
        const double* ct = Ps + (size_t)t * rpc;
        for (int rl = grp; rl < nr; rl += 4)
          if (ra + rl > pr) acc = fma(ck[rl], ct[rl], acc);
      }
      rs[grp * 64 + kk] = acc;
      __syncthreads();
      if (tid < nk) slot(t & 1, g)[tid] = rs[tid] + rs[64 + tid] + rs[128 + tid] + rs[192 + tid];
      if (pr >= ra && pr < ra + nr && tid < nk) *Ri(kRedPiv + (t & 1) * 64 + tid) = Ps[(size_t)(t + tid) * rpc + (pr - ra)];
    }
    if (!grid_sync(a.bar, a.err)) return;
    {
      const int q = t & 1;
      block_sums(
          0, nk, [&](int) { return G; }, [&](int e, int gg) { return __ldcg(Pt(q, gg, e)); },
          [&](int e, double v) { dots[e] = v; });
      if (tid < nk) piv[tid] = __ldcg(Ri(kRedPiv + (t & 1) * 64 + tid));
    }
    __syncthreads();
    if (tid == 0) {
      const double sig = dots[0], alpha = piv[0];
      double tk = 0.0, scal = 0.0, beta = alpha;
      if (sig != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, sig));
        beta = alpha >= 0.0 ? -nrm : nrm;
        tk = (beta - alpha) / beta;
        scal = 1.0 / (alpha - beta);
      }
      misc[0] = tk;
      misc[1] = scal;
      misc[2] = beta;
      taus[t] = tk;
      if (g == 0) a.tau[RBCK(t, a.ntau, a.err)] = tk;
    }
    __syncthreads();
    const double tk = misc[0], scal = misc[1], beta = misc[2];
    if (tk != 0.0) {
      // columns k > t: P(:, k) -= tau v (v^T P(:, k)),  v^T P(:, k) = P(pr, k) + scal d_k
      for (int e = tid; e < nr * (nk - 1); e += kPT) {
        const int rl = e % nr, kq = 1 + e / nr;
        const int r = ra + rl;
        const double wk = fma(scal, dots[kq], piv[kq]);
        double* pk = Ps + (size_t)(t + kq) * rpc + rl;
        if (r > pr) *pk = fma(-tk * wk, Ps[(size_t)t * rpc + rl] * scal, *pk);
        else if (r == pr) *pk = fma(-tk, wk, *pk);
      }
      __syncthreads();
      for (int rl = tid; rl < nr; rl += kPT) {
        const int r = ra + rl;
        double* pt = Ps + (size_t)t * rpc + rl;
        if (r > pr) *pt *= scal;
        else if (r == pr) *pt = beta;
      }
    }
    __syncthreads();
  }
  // the panel back, the new columns of V (values and digits)
  for (int e = tid; e < nr * w; e += kPT) {
    const int rl = e % nr, t = e / nr;
    Pi((size_t)(ra + rl) + (size_t)t * a.ldp) = Ps[t * rpc + rl];
  }
  auto vt = [&](int rl, int t) -> double {
    const int r = ra + rl, pr = a.pv0 + t;
    return r < pr ? 0.0 : (r == pr ? 1.0 : Ps[(size_t)t * rpc + rl]);
  };
  for (int e = tid; e < nr * wp; e += kPT) {
    const int rl = e % nr, t = e / nr;
    const double v = vt(rl, t);
    Vi((size_t)(ra + rl) + (size_t)(j + t) * a.ldv) = v;
    if (v != 0.0) put_digits_v(a.vcol, j + t, ra + rl, v, a.err);
  }
  // S = V(:, 0:j+wp)^T V_s over the panel rows
  const int ns = (j + wp) * wp;
  for (int e = tid; e < ns; e += kPT) {
    const int i = e / wp, t = e % wp;
    double acc = 0.0;
    if (i < j) {
      const size_t v0 = (size_t)ra + (size_t)i * a.ldv;
      for (int rl = 0; rl < nr; ++rl) acc = fma(Vi(v0 + rl), vt(rl, t), acc);
    } else {
      for (int rl = 0; rl < nr; ++rl) acc = fma(vt(rl, i - j), vt(rl, t), acc);
    }
    slot(2, g)[RBCK(e, kPartW, a.err)] = acc;
  }
  if (!grid_sync(a.bar, a.err)) return;
  {
    const int ch = (ns + G - 1) / G;
    block_sums(
        min(ns, g * ch), min(ns, (g + 1) * ch), [&](int) { return G; },
        [&](int e, int gg) { return __ldcg(Pt(2, gg, e)); },
        [&](int e, double v) { *Ri(kRedS + e) = v; });
  }
  if (!grid_sync(a.bar, a.err)) return;
  // T's new columns (Eq. for T, one reflector at a time): row i of CTA i mod G,
  // a warp per row, lanes along k; S and the row staged in shared memory
  double* Ss = Vc;  // ns <= 8192 doubles over Vc and Zs
  for (int e = tid; e < ns; e += kPT) Ss[e] = __ldcg(Ri(kRedS + e));
  __syncthreads();
  double* trow = tw + warp * kBmax;
  for (int i = g + warp * G; i < j + wp; i += 8 * G) {
    for (int k = lane; k < j; k += 32) trow[k] = Ti(i + (size_t)k * kBmax);
    __syncwarp();
    for (int t = 0; t < wp; ++t) {
      const int col = j + t;
      double val;
      if (i > col) {
        val = 0.0;
      } else if (i == col) {
        val = taus[t];
      } else {
        double acc = 0.0;
        for (int k = i + lane; k < col; k += 32) acc = fma(trow[k], Ss[k * wp + t], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        val = -taus[t] * acc;
      }
      __syncwarp();
      if (lane == 0) trow[col] = val;
      __syncwarp();
    }
    for (int t = lane; t < wp; t += 32) Ti(i + (size_t)(j + t) * kBmax) = trow[j + t];
    __syncwarp();
  }
}

// Y's new columns (Eq. for Y): Y(:, j + t) = sum_{t' <= t} (A V_s - Y V^T V_s)(:, t') T_s(t', t)
// for every row of E; A V_s arrives as `ks` partial sums.
__global__ void __launch_bounds__(256) yfix_kernel(const double* __restrict__ AV, int ks, long long kstride,
                                                   long long ldav, int rows, double* __restrict__ Y,
                                                   long long ldy, int j, int wp, const double* __restrict__ S,
                                                   const double* __restrict__ T, size_t nav, size_t ny,
                                                   int* err) {
  extern __shared__ double ysm[];
  double* Ss = ysm;              // S(i, t) for i < j
  double* Tt = Ss + j * wp;      // Tt[t' + t * wp] = T(j + t', j + t)
  const int R = 256 / wp;        // rows per CTA
  double* us = Tt + wp * wp;     // us[t' * R + rl]
  const int tid = threadIdx.x;
  for (int e = tid; e < j * wp; e += 256) Ss[e] = S[RBCK(e, 8192, err)];
  for (int e = tid; e < wp * wp; e += 256)
    Tt[e] = T[RBCK((size_t)(j + e % wp) + (size_t)(j + e / wp) * kBmax, (size_t)kBmax * kBmax, err)];
  __syncthreads();
  const int rl = tid % R, tp = tid / R;
  const int e = blockIdx.x * R + rl;
  const bool act = tp < wp && e < rows;
  if (act) {
    double u = 0.0;
    for (int q = 0; q < ks; ++q) u += AV[RBCK((size_t)q * kstride + e + (size_t)tp * ldav, nav, err)];
    for (int i = 0; i < j; ++i) u = fma(-Y[RBCK(e + (size_t)i * ldy, ny, err)], Ss[i * wp + tp], u);
    us[tp * R + rl] = u;
  }
  __syncthreads();
  if (act) {
    double y = 0.0;
    for (int q = 0; q <= tp; ++q) y = fma(us[q * R + rl], Tt[q + tp * wp], y);
    Y[RBCK(e + (size_t)(j + tp) * ldy, ny, err)] = y;
  }
}

// Z = T^T W for the trailing columns (W in `ks` partial sums, W(i, c) at
// Wp[i + c * kBmax]) straight into Z's digits: operand row c, K = i, with
// the exponent of column c.
__global__ void __launch_bounds__(256) zmake_kernel(const double* __restrict__ Wp, int ks, long long kstride,
                                                    int jb, int cs, int n, const double* __restrict__ T,
                                                    DigitMat Z, size_t nw, int* err) {
  __shared__ double Ws[kBmax][33];
  __shared__ int Es[32];
  const int tid = threadIdx.x;
  const int cb = cs + blockIdx.x * 32;
  for (int e = tid; e < kBmax * 32; e += 256) {
    const int i = e % kBmax, cl = e / kBmax;
    const int c = cb + cl;
    double v = 0.0;
    if (i < jb && c < n)
      for (int q = 0; q < ks; ++q) v += Wp[RBCK((size_t)q * kstride + i + (size_t)c * kBmax, nw, err)];
    Ws[i][cl] = v;
  }
  __syncthreads();
  const int cl = tid & 31, ig = tid >> 5;
  double zv[kBmax / 8];
#pragma unroll
  for (int q = 0; q < kBmax / 8; ++q) {
    const int i = ig + 8 * q;
    double acc = 0.0;
    if (i < jb)
      for (int k = 0; k <= i; ++k) acc = fma(T[RBCK(k + (size_t)i * kBmax, (size_t)kBmax * kBmax, err)], Ws[k][cl], acc);
    zv[q] = acc;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < kBmax / 8; ++q) Ws[ig + 8 * q][cl] = zv[q];
  __syncthreads();
  if (tid < 32) {
    double mx = 0.0;
    for (int i = 0; i < jb; ++i) mx = fmax(mx, fabs(Ws[i][tid]));
    const int E = scale_exp(mx);
    Es[tid] = E;
    if (cb + tid < n) Z.ex[RBCK(cb + tid, (size_t)Z.RT * kTR, err)] = E;
  }
  __syncthreads();
  const int kmax = ((jb + kTK - 1) / kTK) * kTK;
  for (int u = tid; u < 32 * (kBmax / 8); u += 256) {
    const int c2 = u & 31, kg = u >> 5;
    const int c = cb + c2, i0 = kg * 8;
    if (c >= n || i0 >= kmax) continue;
    unsigned short dg[8][kD];
#pragma unroll
    for (int q = 0; q < 8; ++q) digits_of(Ws[i0 + q][c2], Es[c2], dg[q]);
    const size_t off = (size_t)tile_off_kg(c % kTR, i0 % kTK, kTK / 8);
#pragma unroll
    for (int l = 0; l < kD; ++l) {
      uint4 v;
      v.x = (unsigned)dg[0][l] | ((unsigned)dg[1][l] << 16);
      v.y = (unsigned)dg[2][l] | ((unsigned)dg[3][l] << 16);
      v.z = (unsigned)dg[4][l] | ((unsigned)dg[5][l] << 16);
      v.w = (unsigned)dg[6][l] | ((unsigned)dg[7][l] << 16);
      *reinterpret_cast<uint4*>(Z.d + RBCR(tile_index(Z, l, i0 / kTK, c / kTR) + off, 8, Z.nd, err)) = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct RtcScratch {
  double* E;        // (p + n) x n, leading dimension ldE: C above A
  long long ldE;
  double* V;        // ldv x kBmax
  long long ldv;
  double* T;        // kBmax x kBmax
  double* Y;        // ldE x kBmax
  double* W;        // ksW x (kBmax x n)
  double* AV;       // ksY x (ldE x kMaxW)
  double* part;     // 3 x G x kPartW
  double* red;      // kRedTotal
  unsigned* bar;    // [0..3]: [2] the error flag; then one arrival counter per panel launch
  int nbar;         // panel-launch counters available
  int panels;       // panel launches so far
  DigitMat erow, ecol, yrow, vrow, vcol, zcol;
  int G;
  size_t nE, nV, nY, nW, nAV, npart;  // extents in doubles
};

inline long long rup(long long x, long long a) { return (x + a - 1) / a * a; }

size_t digit_bytes(int RT, int KT) { return (size_t)kD * KT * RT * kTileEl * sizeof(unsigned short); }

// Carve (or size, with base == nullptr) the scratch of an n x n reduction.
size_t rtc_layout(int n, int p, unsigned char* base, RtcScratch* S) {
  const int G = std::max(1, num_sms());
  const long long rowsE = (long long)p + n;
  const long long ldE = rup(rowsE, 32), ldv = rup(n, 32);
  const int RTe = 2 * (int)((rowsE + 127) / 128), RTn = 2 * ((n + 127) / 128);
  const int KTn = (n + kTK - 1) / kTK, KTb = kBmax / kTK;
  const int ksW = 8, ksY = 8;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* q = base ? base + off : nullptr;
    off += rup((long long)bytes, 256);
    return q;
  };
  RtcScratch s;
  s.ldE = ldE;
  s.ldv = ldv;
  s.G = G;
  s.nE = (size_t)ldE * n;
  s.nV = (size_t)ldv * kBmax;
  s.nY = (size_t)ldE * kBmax;
  s.nW = (size_t)ksW * kBmax * (size_t)n;
  s.nAV = (size_t)ksY * ldE * kMaxW;
  s.npart = 3 * (size_t)G * kPartW;
  s.E = (double*)take(sizeof(double) * s.nE);
  s.V = (double*)take(sizeof(double) * s.nV);
  s.T = (double*)take(sizeof(double) * kBmax * kBmax);
  s.Y = (double*)take(sizeof(double) * s.nY);
  s.W = (double*)take(sizeof(double) * s.nW);
  s.AV = (double*)take(sizeof(double) * s.nAV);
  s.part = (double*)take(sizeof(double) * s.npart);
  s.red = (double*)take(sizeof(double) * kRedTotal);
  s.nbar = n + 16;
  s.panels = 0;
  s.bar = (unsigned*)take(16 + sizeof(unsigned) * (size_t)s.nbar);
  auto dm = [&](int RT, int KT, bool ex) {
    DigitMat M;
    M.RT = RT;
    M.KT = KT;
    M.d = (unsigned short*)take(digit_bytes(RT, KT));
    M.nd = digit_bytes(RT, KT) / sizeof(unsigned short);
    M.ex = ex ? (int*)take(sizeof(int) * (size_t)RT * kTR) : nullptr;
    return M;
  };
  s.erow = dm(RTe, KTn, true);
  s.ecol = dm(RTn, KTn, true);
  s.yrow = dm(RTe, KTb, true);
  s.vrow = dm(RTn, KTb, true);
  s.vcol = dm(2, KTn, false);
  s.zcol = dm(RTn, KTb, true);
  if (S) *S = s;
  return off;
}

// rows [r_lo, r_hi) x K [k_lo, k_hi) of src into M (tiles of whole 128-row pairs)
int split_into(const double* src, long long sr, long long sk, int r_lo, int r_hi, int k_lo, int k_hi,
               const DigitMat& M, size_t nsrc, int* err, cudaStream_t st) {
  const size_t nex = (size_t)M.RT * kTR;
  if (r_hi <= r_lo || k_hi <= k_lo) return SSV_OK;
  if (M.ex) {
    SSV_CUDA_TRY(cudaMemsetAsync(M.ex, 0x80, sizeof(int) * (size_t)M.RT * kTR, st));
    const int kchunk = 512;
    dim3 grid((unsigned)((r_hi - r_lo + 63) / 64), (unsigned)((k_hi - k_lo + kchunk - 1) / kchunk));
    split_exp_kernel<<<grid, 256, 0, st>>>(src, sr, sk, r_lo, r_hi, k_lo, k_hi, kchunk, M.ex, nsrc, nex, err);
    count_launch();
    SSV_CUDA_TRY(cudaGetLastError());
  }
  const int I0 = 2 * (r_lo / 128), I1 = 2 * ((r_hi + 127) / 128);
  const int J0 = k_lo / kTK, J1 = (k_hi + kTK - 1) / kTK;
  split_dig_kernel<<<dim3((unsigned)(I1 - I0), (unsigned)(J1 - J0)), 256, 0, st>>>(src, sr, sk, r_lo, r_hi, k_lo,
                                                                                 k_hi, M, I0, J0, nsrc, nex, err);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

template <int NT, int LV>
int gemm_launch(const GArgs& g, cudaStream_t st) {
  using Cfg = GCfg<NT, LV>;
  const int nI = (g.M1 + 127) / 128 - g.M0 / 128;
  const int nN = (g.N1 + NT - 1) / NT - g.N0 / NT;
  if (g.M1 <= g.M0 || g.N1 <= g.N0 || nI <= 0 || nN <= 0) return SSV_OK;
  const long long tiles = (long long)nI * nN * g.ksplit;
  const int grid = (int)std::min<long long>(tiles, std::max(1, num_sms()));
  SSV_CUDA_TRY(cudaFuncSetAttribute(tc_gemm_kernel<NT, LV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)Cfg::kSmem));
  tc_gemm_kernel<NT, LV><<<grid, kGT, Cfg::kSmem, st>>>(g);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

// the long-K products (A V_s, V^T A): nine levels, N <= 32
int gemm_long(int width, const GArgs& g, cudaStream_t st) {
  if (width <= 16) return gemm_launch<16, 9>(g, st);
  return gemm_launch<32, 9>(g, st);
}

GArgs gemm_args(const DigitMat& A, const DigitMat& B, int J0, int J1, int M0, int M1, int N0, int N1, double* C,
                size_t nc, long long ldc, int sub, const RtcScratch& S) {
  GArgs g;
  g.seg.A = A;
  g.seg.B = B;
  g.seg.J0 = J0;
  g.seg.J1 = J1;
  g.M0 = M0;
  g.M1 = M1;
  g.N0 = N0;
  g.N1 = N1;
  g.roff = 0;
  g.coff = 0;
  g.C = C;
  g.nc = nc;
  g.ldc = ldc;
  g.sub = sub;
  g.ksplit = 1;
  g.kstride = 0;
  g.err = reinterpret_cast<int*>(S.bar + 2);
  return g;
}

// One mini-block: panel (cooperative), A V_s on the tensor cores, Y's new columns.
int run_panel(RtcScratch& S, int n, int p, double* P, size_t np, long long ldp, int r0, int w, int wp, int pv0,
              int j, int c0, double* tau, size_t ntau, cudaStream_t st) {
  if (S.panels >= S.nbar) return SSV_EINVAL;
  const int L = n - r0;
  int G = std::min(S.G, std::max(1, (L + 15) / 16));
  const int rpc = (L + G - 1) / G;
  if ((long long)rpc * w > kPanRowsW) return SSV_ENOTSUP;
  PanArgs a;
  a.P = P;
  a.ldp = ldp;
  a.r0 = r0;
  a.n = n;
  a.w = w;
  a.wp = wp;
  a.pv0 = pv0;
  a.j = j;
  a.c0 = c0;
  a.V = S.V;
  a.ldv = S.ldv;
  a.T = S.T;
  a.Y = S.Y;
  a.ldy = S.ldE;
  a.yoff = p;
  a.tau = tau;
  a.vcol = S.vcol;
  a.part = S.part;
  a.red = S.red;
  a.bar = S.bar + 4 + S.panels++;
  a.err = reinterpret_cast<int*>(S.bar + 2);
  a.np = np;
  a.nv = S.nV;
  a.ny = S.nY;
  a.ntau = ntau;
  a.npart = S.npart;
  const size_t smem = sizeof(double) * ((size_t)rpc * w + kPanFixed);
  SSV_CUDA_TRY(cudaFuncSetAttribute(panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  void* args[] = {&a};
  SSV_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_kernel, dim3(G), dim3(kPT), args, smem, st));
  count_launch();
  // A V_s: every row of E against the new reflectors (rows pv0.. of V_s are nonzero)
  const int KTn = (n + kTK - 1) / kTK;
  const int rowsE = p + n;
  GArgs g = gemm_args(S.erow, S.vcol, pv0 / kTK, KTn, 0, rowsE, j, j + wp, S.AV, S.nAV, S.ldE, 0, S);
  g.coff = -j;
  const int NT = wp <= 16 ? 16 : 32;
  const int nI = (rowsE + 127) / 128, nN = (j + wp + NT - 1) / NT - j / NT;
  g.ksplit = std::max(1, std::min(8, S.G / std::max(1, nI * nN)));
  g.kstride = S.ldE * kMaxW;
  int rc = gemm_long(wp, g, st);
  if (rc != SSV_OK) return rc;
  const int R = 256 / wp;
  const size_t ysm = sizeof(double) * ((size_t)j * wp + (size_t)wp * wp + 256);
  SSV_CUDA_TRY(cudaFuncSetAttribute(yfix_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm));
  yfix_kernel<<<(rowsE + R - 1) / R, 256, ysm, st>>>(S.AV, g.ksplit, g.kstride, S.ldE, rowsE, S.Y, S.ldE, j, wp,
                                                     S.red + kRedS, S.T, S.nAV, S.nY, a.err);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  return SSV_OK;
}

// Block end (Algorithm 3): right update, W = V^T A, Z = T^T W, left update.
// Rows [0, p + r0) take the right update from column tc0, rows [p + r0, p + n)
// from column cs; the left update covers rows r0.. and columns cs...
int run_block_end(const RtcScratch& S, int n, int p, int r0, int tc0, int cs, int jb, cudaStream_t st) {
  const int rowsE = p + n;
  const int KTn = (n + kTK - 1) / kTK, KTj = (jb + kTK - 1) / kTK;
  int* err = reinterpret_cast<int*>(S.bar + 2);
  int rc = split_into(S.Y, 1, S.ldE, 0, rowsE, 0, jb, S.yrow, S.nY, err, st);
  // V by rows, each with its own exponent (a row of V across the block's
  // reflectors is mostly far below the unit pivots)
  if (rc == SSV_OK) rc = split_into(S.V, 1, S.ldv, 0, n, 0, jb, S.vrow, S.nV, err, st);
  if (rc != SSV_OK) return rc;
  if (tc0 == cs) {
    rc = gemm_launch<64, 8>(gemm_args(S.yrow, S.vrow, 0, KTj, 0, rowsE, cs, n, S.E, S.nE, S.ldE, 1, S), st);
  } else {
    rc = gemm_launch<64, 8>(gemm_args(S.yrow, S.vrow, 0, KTj, 0, p + r0, tc0, n, S.E, S.nE, S.ldE, 1, S), st);
    if (rc == SSV_OK)
      rc = gemm_launch<64, 8>(gemm_args(S.yrow, S.vrow, 0, KTj, p + r0, rowsE, cs, n, S.E, S.nE, S.ldE, 1, S), st);
  }
  if (rc != SSV_OK || cs >= n) return rc;
  rc = split_into(S.E + p, S.ldE, 1, cs, n, r0, n, S.ecol, S.nE - p, err, st);
  if (rc != SSV_OK) return rc;
  GArgs g = gemm_args(S.vcol, S.ecol, r0 / kTK, KTn, 0, jb, cs, n, S.W, S.nW, kBmax, 0, S);
  const int nN = (n + 31) / 32 - cs / 32;
  g.ksplit = std::max(1, std::min(8, S.G / std::max(1, nN)));
  g.kstride = (long long)kBmax * n;
  rc = gemm_launch<32, 9>(g, st);
  if (rc != SSV_OK) return rc;
  zmake_kernel<<<(n - cs + 31) / 32, 256, 0, st>>>(S.W, g.ksplit, g.kstride, jb, cs, n, S.T, S.zcol, S.nW, err);
  count_launch();
  SSV_CUDA_TRY(cudaGetLastError());
  GArgs gl = gemm_args(S.vrow, S.zcol, 0, KTj, r0, n, cs, n, S.E, S.nE, S.ldE, 1, S);
  gl.roff = p;
  return gemm_launch<64, 8>(gl, st);
}

#ifdef SSV_BOUNDS_CHECK
// bit 4 of the error word when a byte of the canary after the scratch changed
__global__ void rtc_canary_kernel(const unsigned char* c, size_t nbytes, int* err) {
  for (size_t i = threadIdx.x; i < nbytes; i += blockDim.x)
    if (c[i] != 0xA5) atomicOr(err, 4);
}
#endif

int clear_block(const RtcScratch& S, int n, cudaStream_t st) {
  SSV_CUDA_TRY(cudaMemsetAsync(S.V, 0, sizeof(double) * S.ldv * kBmax, st));
  SSV_CUDA_TRY(cudaMemsetAsync(S.T, 0, sizeof(double) * kBmax * kBmax, st));
  SSV_CUDA_TRY(cudaMemsetAsync(S.vcol.d, 0, digit_bytes(S.vcol.RT, S.vcol.KT), st));
  (void)n;
  return SSV_OK;
}

}  // namespace

bool reduce_tc_supported(int n, int m) {
  if (m < 1 || m > kMaxW || n < 2) return false;
  const int G = std::max(1, num_sms());
  return (long long)((n + G - 1) / G) * m <= kPanRowsW;
}

size_t reduce_tc_scratch_bytes(int n, int p) { return rtc_layout(n, p, nullptr, nullptr); }

int reduce_tc(Handle* h, cudaStream_t st) {
  const int n = h->n, m = h->m, p = h->p;
  h->kb = std::min(m, n - 1);
  h->ka = std::max(0, n - m - 1);
  if (h->kb <= 0 && h->ka <= 0) return SSV_OK;
  if (!reduce_tc_supported(n, m)) return SSV_ENOTSUP;
  const int ldct = p > 0 ? p : 1;
  const size_t bytes = rtc_layout(n, p, nullptr, nullptr);
#ifdef SSV_BOUNDS_CHECK
  constexpr size_t kCanary = 256;  // checked at the end
#else
  constexpr size_t kCanary = 0;
#endif
  unsigned char* base = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&base, bytes + kCanary, st));
  RtcScratch S;
  rtc_layout(n, p, base, &S);
  int* err = reinterpret_cast<int*>(S.bar + 2);
  int rc = SSV_OK;
  auto step = [&](int r) {
    if (rc == SSV_OK) rc = r;
  };
  auto cu = [&](cudaError_t e) {
    if (rc == SSV_OK && e != cudaSuccess) {
      set_cuda_error(e);
      rc = e == cudaErrorMemoryAllocation ? SSV_ENOMEM : SSV_ECUDA;
    }
  };
#ifdef SSV_BOUNDS_CHECK
  // scratch read before it is written shows up as NaN (0xFF bytes), the canary
  // after the scratch as a changed byte
  cu(cudaMemsetAsync(base, 0xFF, bytes, st));
  cu(cudaMemsetAsync(base + bytes, 0xA5, kCanary, st));
#endif
  cu(cudaMemsetAsync(S.bar, 0, 16 + sizeof(unsigned) * (size_t)S.nbar, st));
  if (p > 0)
    cu(cudaMemcpy2DAsync(S.E, sizeof(double) * S.ldE, h->Ct, sizeof(double) * ldct, sizeof(double) * p, n,
                         cudaMemcpyDeviceToDevice, st));
  cu(cudaMemcpy2DAsync(S.E + p, sizeof(double) * S.ldE, h->H, sizeof(double) * n, sizeof(double) * n, n,
                       cudaMemcpyDeviceToDevice, st));
  // Step 1: the QR of B, applied to A from both sides and to C from the right
  if (h->kb > 0) {
    step(clear_block(S, n, st));
    step(split_into(S.E, 1, S.ldE, 0, p + n, 0, n, S.erow, S.nE, err, st));
    if (rc == SSV_OK)
      step(run_panel(S, n, p, h->R, (size_t)n * m, n, 0, m, h->kb, 0, 0, 0, h->tauB, (size_t)h->kb, st));
    if (rc == SSV_OK) step(run_block_end(S, n, p, 0, 0, 0, h->kb, st));
  }
  // Steps 2-3: the m-Hessenberg reduction of A, blocks of b = floor(128 / m) m columns
  const int b = (kBmax / m) * m;
  for (int z = 0; z < h->ka && rc == SSV_OK; z += b) {
    const int jb = std::min(b, h->ka - z);
    const int r0 = z + m;
    step(clear_block(S, n, st));
    step(split_into(S.E, 1, S.ldE, 0, p + n, r0, n, S.erow, S.nE, err, st));
    for (int j = 0; j < jb && rc == SSV_OK; j += m) {
      const int w = std::min(m, jb - j);
      const int c0 = z + j;
      const size_t off = (size_t)p + (size_t)c0 * S.ldE;
      step(run_panel(S, n, p, S.E + off, S.nE - off, S.ldE, r0, w, w, c0 + m, j, c0, h->tauA + c0,
                     (size_t)(h->ka - c0), st));
    }
    if (rc == SSV_OK) step(run_block_end(S, n, p, r0, r0, z + jb, jb, st));
  }
  cu(cudaMemcpy2DAsync(h->H, sizeof(double) * n, S.E + p, sizeof(double) * S.ldE, sizeof(double) * n, n,
                       cudaMemcpyDeviceToDevice, st));
  if (p > 0)
    cu(cudaMemcpy2DAsync(h->Ct, sizeof(double) * ldct, S.E, sizeof(double) * S.ldE, sizeof(double) * p, n,
                         cudaMemcpyDeviceToDevice, st));
#ifdef SSV_BOUNDS_CHECK
  if (rc == SSV_OK) {
    rtc_canary_kernel<<<1, 256, 0, st>>>(base + bytes, kCanary, err);
    count_launch();
    cu(cudaGetLastError());
  }
#endif
  int herr = 0;
  cu(cudaMemcpyAsync(&herr, S.bar + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
  cu(cudaStreamSynchronize(st));
  // bit 1: a wait gave up; bits 2 and 4 (debug builds): an index out of range,
  // a changed canary
  if (rc == SSV_OK && (herr & 1)) rc = SSV_ETIMEOUT;
  else if (rc == SSV_OK && herr != 0) rc = SSV_ECUDA;
  cudaError_t e2 = cudaFreeAsync(base, st);
  if (e2 != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e2);
    rc = SSV_ECUDA;
  }
  return rc;
}

}  // namespace ssv
