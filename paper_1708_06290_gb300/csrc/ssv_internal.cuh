// Internal declarations of the GB300 shifted-system solver library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ssv.h"

namespace ssv {

// --------------------------------------------------------------------------
// complex double helpers (interleaved re, im)
// --------------------------------------------------------------------------
struct cd {
  double x, y;
};

__host__ __device__ __forceinline__ cd mkcd(double a, double b) { return cd{a, b}; }
__host__ __device__ __forceinline__ cd cadd(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
__host__ __device__ __forceinline__ cd csub(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
__host__ __device__ __forceinline__ cd cmul(cd a, cd b) {
  return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a + b * c
__host__ __device__ __forceinline__ cd cfma(cd b, cd c, cd a) {
  return cd{fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y))};
}
// a - b * c
__host__ __device__ __forceinline__ cd cfms(cd b, cd c, cd a) {
  return cd{fma(-b.x, c.x, fma(b.y, c.y, a.x)), fma(-b.x, c.y, fma(-b.y, c.x, a.y))};
}
__host__ __device__ __forceinline__ double cabs1(cd a) { return fabs(a.x) + fabs(a.y); }
// a / b (Smith's algorithm, Smith 1962)
__host__ __device__ __forceinline__ cd cdiv(cd a, cd b) {
  if (fabs(b.y) <= fabs(b.x)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return cd{(a.x + a.y * r) / d, (a.y - a.x * r) / d};
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return cd{(a.x * r + a.y) / d, (a.y * r - a.x) / d};
  }
}

// --------------------------------------------------------------------------
// handle
// --------------------------------------------------------------------------
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

struct Handle {
  int n, m, p;
  int dev;
  double* H;      // n x n, ld n; Householder vectors of Q_A below the m-th subdiagonal
  double* R;      // n x m, ld n; Householder vectors of Q_B below the diagonal
  double* Ct;     // max(p,1) x n, ld max(p,1)
  double* tauB;   // m
  double* tauA;   // n
  double* hnorm2; // 2: ||H||_F^2 and trace(H) of the structural part
  float* Hhi;     // n x n: fl32(H) on and above the m-th subdiagonal, 0 below
  float* Hlo;     // n x n: fl32(H - Hhi), 0 below (Hhi + Hlo carries 48 bits of H)
  int kb;         // number of Q_B reflectors
  int ka;         // number of Q_A reflectors
  int has_q;      // 0 when built by ssv_load_reduced
  size_t bytes;
};

// error plumbing (thread-local last CUDA error)
void set_cuda_error(cudaError_t e);
// stream-ordered device allocation from the library's memory pool on the
// current device (freed with cudaFreeAsync); the pool keeps freed blocks for
// reuse instead of returning them at every synchronisation (ssv_pool_trim)
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st);
#define SSV_CUDA_TRY(expr)                         \
  do {                                             \
    cudaError_t _e = (expr);                       \
    if (_e != cudaSuccess) {                       \
      ::ssv::set_cuda_error(_e);                   \
      return _e == cudaErrorMemoryAllocation ? SSV_ENOMEM : SSV_ECUDA; \
    }                                              \
  } while (0)

// the reduction proper: one persistent cooperative kernel (reduce_persistent.cu);
// H, R, Ct hold copies of A, B, C on entry.  Synchronises `st`.
int reduce_persistent(Handle* h, cudaStream_t st);
// self-test of the bounded grid barrier (expects SSV_ETIMEOUT)
int barrier_selftest(long long limit, cudaStream_t st);
// the reduction with two levels of blocking and its O(n^3) products as
// FP64-accurate BF16 digit products on the tensor cores (reduce_tc.cu); same
// contract as reduce_persistent.  Synchronises `st`.
int reduce_tc(Handle* h, cudaStream_t st);
bool reduce_tc_supported(int n, int m);
size_t reduce_tc_scratch_bytes(int n, int p);
// reduction (reduce_fp64.cu): arith SSV_REDUCE_FP64 or SSV_REDUCE_TENSOR
int reduce_fp64(Handle* h, const double* A, long long lda, const double* B, long long ldb,
                const double* C, long long ldc, int arith, cudaStream_t st);
// back-transform X = Q Xhat (reduce_fp64.cu)
int apply_q_fp64(const Handle* h, int ncols, const double* Xhat, long long ldx, double* X,
                 long long ldX, cudaStream_t st);
// load a stored reduced triple with explicit zeros (reduce_fp64.cu)
int load_reduced(Handle* h, const double* H, long long ldh, const double* R, long long ldr,
                 const double* Ct, long long ldc, cudaStream_t st);
// copy-out with explicit zeros (reduce_fp64.cu)
int get_reduced(const Handle* h, double* H, long long ldh, double* R, long long ldr, double* Ct,
                long long ldc, cudaStream_t st);

// solver (solve_fp64.cu)
int solve_fp64(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
               long long ldo, int* status, double* resid, cudaStream_t st);
// one right-hand side B bhat_l per shift (Sec. 3.3); mode G / TF / XHAT (X = XHAT
// here, the caller applies Q)
int solve_fp64_rhs(const Handle* h, int s, const double* shifts, const double* bhat,
                   long long ldb, const ssv_opts* o, double* out, long long ldo, int* status,
                   cudaStream_t st);
// transposed systems (A - sigma_l I)^T x_l = C^T chat_l (Sec. 3.3); out = Q^T x_l (n x s)
int solve_fp64_trans(const Handle* h, int s, const double* shifts, const double* chat,
                     long long ldc, const ssv_opts* o, double* out, long long ldo, int* status,
                     cudaStream_t st);
// FP64 sweep with the Givens panel and greedy schedule (Sec. 3.2); n_b <= 32
int solve_fp64_givens(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                      long long ldo, int* status, double* resid, cudaStream_t st);
// ||C (sigma I - A)^{-1} B||_2 per shift (structured pseudospectra, Sec. 1), tf_norm.cu
int tf_norm2(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* norms,
             int* status, cudaStream_t st);
// greedy annihilation schedule (Algorithm 9) of a block with `rows` rows and rows + m
// columns: rotations packed r | c1 << 8 | c2 << 16 (0-based), step t = off[t] .. off[t+1]-1
void greedy_rows(int rows, int m, std::vector<int>* rot, std::vector<int>* off);
// FP64 solve restricted to the shifts with mask[j] != 0 (others untouched)
int solve_fp64_masked(const Handle* h, int s, const double* shifts, int mode, int nb,
                      double* out, long long ldo, int* status, const int* mask, void* xhat_copy,
                      long long ldxc, cudaStream_t st);
// mixed-precision solve with FP64-accurate refinement (solve_mixed.cu)
int solve_mixed(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                long long ldo, int* status, double* resid, cudaStream_t st);
size_t solve_mixed_scratch_bytes(int n, int m, int p, int s, const ssv_opts* o);
// refinement counters of the mixed path on the current device: c[0] correction
// shift-sweeps, c[1] FP64 re-solves (synchronising read, optional reset)
int refine_counts(long long c[2], bool reset);
// split H into the FP32 pair (Hhi, Hlo) (reduce_fp64.cu)
int split_h(Handle* h, cudaStream_t st);
size_t solve_fp64_scratch_bytes(int n, int m, int p, int s, const ssv_opts* o);
// normwise backward error of computed Xhat (residual_fp64.cu)
int backward_error_fp64(const Handle* h, int s, const double* shifts, const double* Xhat,
                        long long ldx, double* resid, cudaStream_t st);
// same, only for the shifts with mask[j] != 0
int backward_error_fp64_masked(const Handle* h, int s, const double* shifts, const double* Xhat,
                               long long ldx, double* resid, const int* mask, cudaStream_t st);

// FP64-accurate residual on the tensor cores (residual_tc.cu): Ozaki-split
// BF16 digit slices of H (per row) and Xhat (per real column), m <= kTcMaxM.
constexpr int kTcMaxM = 16;
int resid_tc_npad(int n);
size_t resid_tc_hbytes(int n);
size_t resid_tc_xbytes(int n, int s);
int resid_tc_split_h(const Handle* h, void* hbuf, cudaStream_t st);
// E (complex64, n x m per shift, may be null) and acc += (||E||_F^2, ||Xhat||_F^2)
// for the shifts list[0 .. *count); Xhat of shift j at Xhat + 2 j m ldx doubles
int resid_tc_run(const Handle* h, const void* hbuf, void* xbuf, int s, const double* shifts,
                 const int* list, const int* count, const double* Xhat, long long ldx, void* E,
                 double* acc, int* err, cudaStream_t st);
// K depth of one H digit tile (columns per tile of the layout above)
int resid_tc_ktile();
// the sweep with the Z1 P1 update on the tensor cores (solve_tc.cu): m <= 16,
// n > m, modes G / TF / XHAT; hdig = H digit tiles from resid_tc_split_h, or
// null to split here
bool solve_tc_supported(const Handle* h, int mode);
size_t solve_tc_scratch_bytes(int n, int m, int p, int s, int mode);
int solve_tc(const Handle* h, int s, const double* shifts, int mode, double* out, long long ldo,
             int* status, const void* hdig, cudaStream_t st);
// SSV_SPLIT solve (ssv_api.cu): the tensor-core sweep, optional FP64 backward errors
int solve_split(const Handle* h, int s, const double* shifts, int mode, double* out, long long ldo,
                int* status, double* resid, cudaStream_t st);
// normwise backward error of computed Xhat with the tensor-core residual
int backward_error_tc(const Handle* h, int s, const double* shifts, const double* Xhat,
                      long long ldx, double* eta, cudaStream_t st);

// allocation-free FP64 solve on the library's fixed scratch array (solve_fp64.cu)
int solve_fp64_noalloc(const Handle* h, int s, const double* shifts, const ssv_opts* o,
                       double* out, long long ldo, int* status, cudaStream_t st);
size_t noalloc_scratch_bytes();

int default_nb(int n, int m);
int num_sms();

// batched multi-system FP64 solve (solve_fp64.cu)
struct BatchPlan;
// stream_ordered != nullptr: stream-ordered buffers on that stream (freed by
// batch_destroy on it, no device-wide synchronisation); else cudaMalloc.
int batch_create(int nsys, const Handle* const* hs, const int* s, const double* const* shifts,
                 const ssv_opts* o, double* const* outs, const long long* ldos, int* const* status,
                 BatchPlan** out, cudaStream_t stream_ordered);
int batch_run(const BatchPlan* bp, cudaStream_t st);
void batch_destroy(BatchPlan* bp);
// n_b autotuner (solve_fp64.cu)
int tuned_nb(int n, int m, int p, int prec, int mode);
int autotune_nb(const Handle* h, int s, const double* shifts, const ssv_opts* o, double* out,
                long long ldo, cudaStream_t st, int* best_nb, float* best_ms);

// Phase tracer (trace.cu): no-ops unless enabled with ssv_trace_enable.
bool trace_on();
void* trace_begin(const char* name, cudaStream_t st);
void trace_end(void* tok, cudaStream_t st);

// Kernel-launch counter (every launch site calls count_launch()).
void count_launch(long long k = 1);
// DFMA (kind 0) / FFMA (kind 1) throughput probe, TFLOP/s.
int peak_probe(int kind, cudaStream_t st, double* tflops);

}  // namespace ssv
