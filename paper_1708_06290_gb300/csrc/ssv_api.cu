// C ABI entry points (include/ssv.h): argument checks, handle lifetime and
// dispatch to the FP64 reduction and the solvers.
#include <atomic>
#include <mutex>
#include <cstdlib>
#include <cstring>
#include <new>

#include "ssv_internal.cuh"

namespace ssv {

static thread_local int g_last_cuda = 0;
static std::atomic<long long> g_launches{0};

void set_cuda_error(cudaError_t e) { g_last_cuda = (int)e; }

// One memory pool per device for the library's stream-ordered scratch.  The
// device's default pool hands freed memory back at every synchronisation, so
// a solve after a synchronisation maps its (up to tens of GB of) scratch anew;
// this pool keeps what it has mapped (release threshold: no limit) until
// ssv_pool_trim.
namespace {
constexpr int kMaxPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
}  // namespace

static cudaError_t device_pool(cudaMemPool_t* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxPoolDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (g_pool[dev] == nullptr) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    e = cudaMemPoolCreate(&pool, &props);
    if (e != cudaSuccess) return e;
    unsigned long long keep = ~0ull;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
      cudaMemPoolDestroy(pool);
      return e;
    }
    g_pool[dev] = pool;
  }
  *out = g_pool[dev];
  return cudaSuccess;
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t st) {
  cudaMemPool_t pool = nullptr;
  cudaError_t e = device_pool(&pool);
  if (e != cudaSuccess) return e;
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}
void count_launch(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 132;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 132;
    cached[dev] = v;
  }
  return cached[dev];
}

static void free_handle_buffers(Handle* h) {
  if (!h) return;
  cudaFree(h->H);
  cudaFree(h->R);
  cudaFree(h->Ct);
  cudaFree(h->tauB);
  cudaFree(h->tauA);
  cudaFree(h->hnorm2);
  cudaFree(h->Hhi);
  cudaFree(h->Hlo);
}

static size_t handle_bytes(int n, int m, int p) {
  size_t b = sizeof(double) * ((size_t)n * n + (size_t)n * m + (size_t)(p > 0 ? p : 1) * n +
                               (size_t)m + (size_t)n + 2) +
             2 * sizeof(float) * (size_t)n * n;
  return b;
}

static int check_opts(const ssv_opts* o) {
  if (o->precision != SSV_FP64 && o->precision != SSV_MIXED && o->precision != SSV_DFLOAT &&
      o->precision != SSV_SPLIT)
    return SSV_EINVAL;
  if (o->mode < SSV_G || o->mode > SSV_X) return SSV_EINVAL;
  if (o->nb < 0 || o->max_refine < 0 || !(o->tol >= 0.0)) return SSV_EINVAL;
  if (o->panel != SSV_PANEL_HOUSEHOLDER && o->panel != SSV_PANEL_GIVENS) return SSV_EINVAL;
  if (o->first != SSV_FIRST_DFLOAT && o->first != SSV_FIRST_C64 && o->first != SSV_FIRST_TENSOR)
    return SSV_EINVAL;
  return SSV_OK;
}

// SSV_SPLIT: the tensor-core sweep; with resid, the backward errors come from
// the FP64 residual of X-hat (solved once more in X-hat mode for G / TF)
int solve_split(const Handle* h, int s, const double* shifts, int mode, double* out, long long ldo,
                int* status, double* resid, cudaStream_t st) {
  if (!solve_tc_supported(h, mode)) return SSV_ENOTSUP;
  void* tr = trace_begin("solve_split", st);
  int rc = solve_tc(h, s, shifts, mode, out, ldo, status, nullptr, st);
  trace_end(tr, st);
  if (rc != SSV_OK || resid == nullptr) return rc;
  if (mode == SSV_XHAT) return backward_error_fp64(h, s, shifts, out, ldo, resid, st);
  double* xc = nullptr;
  SSV_CUDA_TRY(pool_alloc((void**)&xc, sizeof(double) * 2 * (size_t)h->n * h->m * s, st));
  rc = solve_tc(h, s, shifts, SSV_XHAT, xc, h->n, nullptr, nullptr, st);
  if (rc == SSV_OK) rc = backward_error_fp64(h, s, shifts, xc, h->n, resid, st);
  cudaError_t e = cudaFreeAsync(xc, st);
  if (e != cudaSuccess && rc == SSV_OK) {
    set_cuda_error(e);
    rc = SSV_ECUDA;
  }
  return rc;
}

}  // namespace ssv

using namespace ssv;

extern "C" {

void ssv_default_opts(ssv_opts* o) {
  if (!o) return;
  o->precision = SSV_FP64;
  o->mode = SSV_G;
  o->nb = 0;
  o->max_refine = 8;
  o->tol = 1e-13;
  o->panel = SSV_PANEL_HOUSEHOLDER;
  o->first = SSV_FIRST_TENSOR;
}

static int make_handle(int n, int m, int p, cudaStream_t st, Handle** out) {
  Handle* h = new (std::nothrow) Handle();
  if (!h) return SSV_ENOMEM;
  std::memset(h, 0, sizeof(Handle));
  h->n = n;
  h->m = m;
  h->p = p;
  cudaGetDevice(&h->dev);
  const int ldct = p > 0 ? p : 1;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](double** ptr, size_t count) {
    if (e == cudaSuccess) e = cudaMalloc((void**)ptr, sizeof(double) * (count ? count : 1));
  };
  alloc(&h->H, (size_t)n * n);
  alloc(&h->R, (size_t)n * m);
  alloc(&h->Ct, (size_t)ldct * n);
  alloc(&h->tauB, (size_t)m);
  alloc(&h->tauA, (size_t)n);
  alloc(&h->hnorm2, 2);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->Hhi, sizeof(float) * (size_t)n * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->Hlo, sizeof(float) * (size_t)n * n);
  if (e == cudaSuccess && p == 0) e = cudaMemsetAsync(h->Ct, 0, sizeof(double) * n, st);
  if (e != cudaSuccess) {
    set_cuda_error(e);
    free_handle_buffers(h);
    delete h;
    return e == cudaErrorMemoryAllocation ? SSV_ENOMEM : SSV_ECUDA;
  }
  h->bytes = handle_bytes(n, m, p);
  *out = h;
  return SSV_OK;
}

int ssv_reduce(int n, int m, int p, const double* A, long long lda, const double* B,
               long long ldb, const double* C, long long ldc, void* stream, ssv_handle* out) {
  return ssv_reduce_arith(n, m, p, A, lda, B, ldb, C, ldc, SSV_REDUCE_FP64, stream, out);
}

int ssv_reduce_arith(int n, int m, int p, const double* A, long long lda, const double* B,
                     long long ldb, const double* C, long long ldc, int arith, void* stream,
                     ssv_handle* out) {
  if (!out) return SSV_EINVAL;
  if (arith != SSV_REDUCE_FP64 && arith != SSV_REDUCE_TENSOR) return SSV_EINVAL;
  *out = nullptr;
  if (n < 1 || m < 1 || m > n || p < 0) return SSV_EINVAL;
  if (!A || !B || (p > 0 && !C)) return SSV_EINVAL;
  if (lda < n || ldb < n || (p > 0 && ldc < p)) return SSV_EINVAL;
  if (arith == SSV_REDUCE_TENSOR && !reduce_tc_supported(n, m)) return SSV_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  Handle* h = nullptr;
  int rc = make_handle(n, m, p, st, &h);
  if (rc != SSV_OK) return rc;
  void* tr = trace_begin(arith == SSV_REDUCE_TENSOR ? "reduce_tc" : "reduce", st);
  rc = reduce_fp64(h, A, lda, B, ldb, C, ldc, arith, st);
  if (rc == SSV_OK) rc = split_h(h, st);
  trace_end(tr, st);
  if (rc != SSV_OK) {
    cudaStreamSynchronize(st);
    free_handle_buffers(h);
    delete h;
    return rc;
  }
  *out = reinterpret_cast<ssv_handle>(h);
  return SSV_OK;
}

int ssv_load_reduced(int n, int m, int p, const double* H, long long ldh, const double* R,
                     long long ldr, const double* Ct, long long ldc, void* stream,
                     ssv_handle* out) {
  if (!out) return SSV_EINVAL;
  *out = nullptr;
  if (n < 1 || m < 1 || m > n || p < 0) return SSV_EINVAL;
  if (!H || !R || (p > 0 && !Ct)) return SSV_EINVAL;
  if (ldh < n || ldr < n || (p > 0 && ldc < p)) return SSV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Handle* h = nullptr;
  int rc = make_handle(n, m, p, st, &h);
  if (rc != SSV_OK) return rc;
  rc = load_reduced(h, H, ldh, R, ldr, Ct, ldc, st);
  if (rc == SSV_OK) rc = split_h(h, st);
  if (rc != SSV_OK) {
    cudaStreamSynchronize(st);
    free_handle_buffers(h);
    delete h;
    return rc;
  }
  *out = reinterpret_cast<ssv_handle>(h);
  return SSV_OK;
}

int ssv_solve(ssv_handle hh, int s, const double* shifts, const ssv_opts* o_in, double* out,
              long long ldo, int* status, double* resid, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 0) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (s == 0) return SSV_OK;
  if (!shifts || !out) return SSV_EINVAL;
  const bool gmode = (o.mode == SSV_G || o.mode == SSV_TF);
  if (gmode && ldo < (h->p > 0 ? h->p : 1)) return SSV_EINVAL;
  if (!gmode && ldo < h->n) return SSV_EINVAL;
  if (o.mode == SSV_X && !h->has_q) return SSV_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  if (o.panel == SSV_PANEL_GIVENS) {
    if (o.precision != SSV_FP64) return SSV_ENOTSUP;
    void* tr = trace_begin("solve_fp64_givens", st);
    rc = solve_fp64_givens(h, s, shifts, &o, out, ldo, status, resid, st);
    trace_end(tr, st);
  } else if (o.precision == SSV_MIXED) {
    rc = solve_mixed(h, s, shifts, &o, out, ldo, status, resid, st);
  } else if (o.precision == SSV_SPLIT) {
    rc = solve_split(h, s, shifts, o.mode == SSV_X ? SSV_XHAT : o.mode, out, ldo, status, resid, st);
  } else {
    void* tr = trace_begin(o.precision == SSV_DFLOAT ? "solve_dfloat" : "solve_fp64", st);
    rc = solve_fp64(h, s, shifts, &o, out, ldo, status, resid, st);
    trace_end(tr, st);
  }
  if (rc == SSV_OK && o.mode == SSV_X) rc = apply_q_fp64(h, s * h->m, out, ldo, out, ldo, st);
  return rc;
}

int ssv_solve_rhs(ssv_handle hh, int s, const double* shifts, const double* bhat, long long ldb,
                  const ssv_opts* o_in, double* out, long long ldo, int* status, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 0) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.precision != SSV_FP64) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  if (!shifts || !out || !bhat || ldb < h->m) return SSV_EINVAL;
  const bool gmode = (o.mode == SSV_G || o.mode == SSV_TF);
  if (gmode && ldo < (h->p > 0 ? h->p : 1)) return SSV_EINVAL;
  if (!gmode && ldo < h->n) return SSV_EINVAL;
  if (o.mode == SSV_X && !h->has_q) return SSV_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  void* tr = trace_begin("solve_rhs", st);
  rc = solve_fp64_rhs(h, s, shifts, bhat, ldb, &o, out, ldo, status, st);
  trace_end(tr, st);
  if (rc == SSV_OK && o.mode == SSV_X) rc = apply_q_fp64(h, s, out, ldo, out, ldo, st);
  return rc;
}

int ssv_solve_trans(ssv_handle hh, int s, const double* shifts, const double* chat, long long ldc,
                    const ssv_opts* o_in, double* out, long long ldo, int* status, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 0) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.precision != SSV_FP64) return SSV_ENOTSUP;
  if (o.mode != SSV_X && o.mode != SSV_XHAT) return SSV_ENOTSUP;
  if (h->p < 1) return SSV_EINVAL;
  if (s == 0) return SSV_OK;
  if (!shifts || !out || !chat || ldc < h->p || ldo < h->n) return SSV_EINVAL;
  if (o.mode == SSV_X && !h->has_q) return SSV_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  void* tr = trace_begin("solve_trans", st);
  rc = solve_fp64_trans(h, s, shifts, chat, ldc, &o, out, ldo, status, st);
  trace_end(tr, st);
  if (rc == SSV_OK && o.mode == SSV_X) rc = apply_q_fp64(h, s, out, ldo, out, ldo, st);
  return rc;
}

int ssv_givens_schedule(int rows, int m, int* rot, int max_rot, int* off, int max_steps,
                        int* nsteps) {
  if (rows < 1 || m < 1 || rows > 255 || rows + m > 255 || !rot || !off || !nsteps) return SSV_EINVAL;
  std::vector<int> r, o;
  greedy_rows(rows, m, &r, &o);
  const int ns = (int)o.size() - 1;
  if ((int)r.size() > max_rot || ns > max_steps) return SSV_EINVAL;
  for (size_t j = 0; j < r.size(); ++j) {
    rot[3 * j] = (r[j] & 255) + 1;
    rot[3 * j + 1] = ((r[j] >> 8) & 255) + 1;
    rot[3 * j + 2] = ((r[j] >> 16) & 255) + 1;
  }
  for (int t = 0; t <= ns; ++t) off[t] = o[t];
  *nsteps = ns;
  return (int)r.size();
}

int ssv_tf_norm2(ssv_handle hh, int s, const double* shifts, const ssv_opts* o_in, double* norms,
                 int* status, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 0) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.panel != SSV_PANEL_HOUSEHOLDER) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  if (!shifts || !norms) return SSV_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  void* tr = trace_begin("tf_norm2", st);
  rc = tf_norm2(h, s, shifts, &o, norms, status, st);
  trace_end(tr, st);
  return rc;
}

int ssv_backward_error(ssv_handle hh, int s, const double* shifts, const double* xhat,
                       long long ldx, int method, double* eta, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 0 || ldx < h->n) return SSV_EINVAL;
  if (method != SSV_RESID_FP64 && method != SSV_RESID_TENSOR) return SSV_EINVAL;
  if (s == 0) return SSV_OK;
  if (!shifts || !xhat || !eta) return SSV_EINVAL;
  if (method == SSV_RESID_TENSOR && h->m > kTcMaxM) return SSV_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  void* tr = trace_begin("backward_error", st);
  const int rc = method == SSV_RESID_TENSOR ? backward_error_tc(h, s, shifts, xhat, ldx, eta, st)
                                            : backward_error_fp64(h, s, shifts, xhat, ldx, eta, st);
  trace_end(tr, st);
  return rc;
}

static int check_many(int nsys, const ssv_handle* hs, const int* s, const double* const* shifts,
                      const ssv_opts& o, double* const* outs, const long long* ldos) {
  if (nsys < 0 || (nsys > 0 && (!hs || !s || !shifts || !outs || !ldos))) return SSV_EINVAL;
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.mode == SSV_X) return SSV_ENOTSUP;
  int dev = 0;
  cudaGetDevice(&dev);
  for (int k = 0; k < nsys; ++k) {
    const Handle* h = reinterpret_cast<const Handle*>(hs[k]);
    if (!h || s[k] < 0) return SSV_EINVAL;
    if (h->dev != dev) return SSV_EINVAL;
    if (s[k] > 0 && (!shifts[k] || !outs[k])) return SSV_EINVAL;
    const bool gmode = (o.mode == SSV_G || o.mode == SSV_TF);
    if (gmode && ldos[k] < (h->p > 0 ? h->p : 1)) return SSV_EINVAL;
    if (!gmode && ldos[k] < h->n) return SSV_EINVAL;
  }
  return SSV_OK;
}

int ssv_solve_many(int nsys, const ssv_handle* hs, const int* s, const double* const* shifts,
                   const ssv_opts* o_in, double* const* outs, const long long* ldos,
                   int* const* status, void* stream) {
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_many(nsys, hs, s, shifts, o, outs, ldos);
  if (rc != SSV_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (o.precision == SSV_MIXED || o.precision == SSV_SPLIT) {
    for (int k = 0; k < nsys && rc == SSV_OK; ++k) {
      const Handle* hk = reinterpret_cast<const Handle*>(hs[k]);
      int* stk = status ? status[k] : nullptr;
      rc = o.precision == SSV_MIXED
               ? solve_mixed(hk, s[k], shifts[k], &o, outs[k], ldos[k], stk, nullptr, st)
               : solve_split(hk, s[k], shifts[k], o.mode, outs[k], ldos[k], stk, nullptr, st);
    }
    return rc;
  }
  // stream-ordered plan on a non-default stream (no device-wide synchronisation);
  // on the legacy default stream the plan is ordinary and freed after a sync
  BatchPlan* bp = nullptr;
  cudaStream_t so = st != nullptr ? st : nullptr;
  rc = batch_create(nsys, reinterpret_cast<const Handle* const*>(hs), s, shifts, &o, outs, ldos,
                    status, &bp, so);
  if (rc != SSV_OK) return rc;
  void* tr = trace_begin("batch", st);
  rc = batch_run(bp, st);
  trace_end(tr, st);
  if (so == nullptr) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && rc == SSV_OK) { set_cuda_error(e); rc = SSV_ECUDA; }
  }
  batch_destroy(bp);
  return rc;
}

int ssv_batch_create(int nsys, const ssv_handle* hs, const int* s, const double* const* shifts,
                     const ssv_opts* o_in, double* const* outs, const long long* ldos,
                     int* const* status, ssv_batch* out) {
  if (!out) return SSV_EINVAL;
  *out = nullptr;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_many(nsys, hs, s, shifts, o, outs, ldos);
  if (rc != SSV_OK) return rc;
  if (o.precision == SSV_MIXED || o.precision == SSV_SPLIT) return SSV_ENOTSUP;
  BatchPlan* bp = nullptr;
  rc = batch_create(nsys, reinterpret_cast<const Handle* const*>(hs), s, shifts, &o, outs, ldos,
                    status, &bp, nullptr);
  if (rc == SSV_OK) *out = reinterpret_cast<ssv_batch>(bp);
  return rc;
}

int ssv_batch_run(ssv_batch b, void* stream) {
  if (!b) return SSV_EINVAL;
  return batch_run(reinterpret_cast<BatchPlan*>(b), (cudaStream_t)stream);
}

void ssv_batch_destroy(ssv_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_destroy(reinterpret_cast<BatchPlan*>(b));
}

int ssv_autotune(ssv_handle hh, int s, const double* shifts, const ssv_opts* o_in, double* out,
                 long long ldo, void* stream, int* best_nb, float* best_ms) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 1 || !shifts || !out || !best_nb) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.mode == SSV_X || o.precision == SSV_SPLIT) return SSV_ENOTSUP;  // SSV_SPLIT: n_b = 128
  const bool gmode = (o.mode == SSV_G || o.mode == SSV_TF);
  if (gmode && ldo < (h->p > 0 ? h->p : 1)) return SSV_EINVAL;
  if (!gmode && ldo < h->n) return SSV_EINVAL;
  return autotune_nb(h, s, shifts, &o, out, ldo, (cudaStream_t)stream, best_nb, best_ms);
}

int ssv_solve_noalloc(ssv_handle hh, int s, const double* shifts, const ssv_opts* o_in,
                      double* out, long long ldo, int* status, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || s < 0) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.precision != SSV_FP64 || o.mode == SSV_X) return SSV_ENOTSUP;
  if (o.panel != SSV_PANEL_HOUSEHOLDER) return SSV_ENOTSUP;
  if (h->m > 32) return SSV_ENOTSUP;
  if (s == 0) return SSV_OK;
  if (!shifts || !out) return SSV_EINVAL;
  const bool gmode = (o.mode == SSV_G || o.mode == SSV_TF);
  if (gmode && ldo < (h->p > 0 ? h->p : 1)) return SSV_EINVAL;
  if (!gmode && ldo < h->n) return SSV_EINVAL;
  return solve_fp64_noalloc(h, s, shifts, &o, out, ldo, status, (cudaStream_t)stream);
}

int ssv_apply_q(ssv_handle hh, int ncols, const double* Xhat, long long ldx, double* X,
                long long ldX, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h || ncols < 0) return SSV_EINVAL;
  if (ncols == 0) return SSV_OK;
  if (!Xhat || !X || ldx < h->n || ldX < h->n) return SSV_EINVAL;
  if (!h->has_q) return SSV_ENOTSUP;
  return apply_q_fp64(h, ncols, Xhat, ldx, X, ldX, (cudaStream_t)stream);
}

int ssv_get_reduced(ssv_handle hh, double* H, long long ldh, double* R, long long ldr, double* Ct,
                    long long ldc, void* stream) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return SSV_EINVAL;
  if ((H && ldh < h->n) || (R && ldr < h->n) || (Ct && h->p > 0 && ldc < h->p)) return SSV_EINVAL;
  return get_reduced(h, H, ldh, R, ldr, Ct, ldc, (cudaStream_t)stream);
}

int ssv_dims(ssv_handle hh, int* n, int* m, int* p) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return SSV_EINVAL;
  if (n) *n = h->n;
  if (m) *m = h->m;
  if (p) *p = h->p;
  return SSV_OK;
}

int ssv_footprint(int n, int m, int p, int s, const ssv_opts* o_in, size_t* bytes) {
  if (!bytes || n < 1 || m < 1 || m > n || p < 0 || s < 0) return SSV_EINVAL;
  ssv_opts o;
  if (o_in) o = *o_in; else ssv_default_opts(&o);
  int rc = check_opts(&o);
  if (rc != SSV_OK) return rc;
  if (o.precision == SSV_SPLIT)
    *bytes = solve_tc_scratch_bytes(n, m, p, s, o.mode == SSV_X ? SSV_XHAT : o.mode) +
             resid_tc_hbytes(n);
  else
    *bytes = o.precision == SSV_MIXED ? solve_mixed_scratch_bytes(n, m, p, s, &o)
                                      : solve_fp64_scratch_bytes(n, m, p, s, &o);
  return SSV_OK;
}

int ssv_handle_bytes(int n, int m, int p, size_t* bytes) {
  if (!bytes || n < 1 || m < 1 || m > n || p < 0) return SSV_EINVAL;
  *bytes = handle_bytes(n, m, p);
  return SSV_OK;
}

void ssv_destroy(ssv_handle hh) {
  Handle* h = reinterpret_cast<Handle*>(hh);
  if (!h) return;
  cudaDeviceSynchronize();
  free_handle_buffers(h);
  delete h;
}

const char* ssv_strerror(int code) {
  switch (code) {
    case SSV_OK: return "success";
    case SSV_EINVAL: return "invalid argument";
    case SSV_ENOMEM: return "device memory allocation failed";
    case SSV_ECUDA: return "CUDA runtime error";
    case SSV_ETIMEOUT: return "bounded device wait timed out";
    case SSV_ENOTSUP: return "unsupported option combination";
    case SSV_ESCRATCH: return "problem exceeds the fixed 64 MiB scratch of ssv_solve_noalloc";
    default: return "unknown error code";
  }
}

int ssv_last_cuda_error(void) { return g_last_cuda; }

int ssv_pool_trim(size_t keep_bytes) {
  cudaMemPool_t pool = nullptr;
  SSV_CUDA_TRY(device_pool(&pool));
  SSV_CUDA_TRY(cudaMemPoolTrimTo(pool, keep_bytes));
  return SSV_OK;
}

int ssv_refine_counts(long long* corrections, long long* resolves, int reset) {
  long long c[2] = {0, 0};
  const int rc = refine_counts(c, reset != 0);
  if (rc != SSV_OK) return rc;
  if (corrections) *corrections = c[0];
  if (resolves) *resolves = c[1];
  return SSV_OK;
}

long long ssv_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

int ssv_selftest_barrier(long long spin_limit, void* stream) {
  if (spin_limit < 1) return SSV_EINVAL;
  return barrier_selftest(spin_limit, (cudaStream_t)stream);
}

int ssv_peak_probe(int kind, void* stream, double* tflops) {
  if (!tflops || (kind != 0 && kind != 1)) return SSV_EINVAL;
  return peak_probe(kind, (cudaStream_t)stream, tflops);
}

}  // extern "C"
