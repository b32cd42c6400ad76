// fwi_runtime.cu -- host runtime and C ABI of the full-space Gauss-Newton FWI
// library (see include/fwikkt.h for the entry points and their contracts).
//
// Everything numerical runs in the kernels of fwi_kernels.cuh; this file owns
// device memory, builds the descriptor tables of the batch (blocks, operators,
// row tiles, multigrid levels), sequences the kernel launches of the solvers
// and reads back only scalars (residual norms) to steer the iterations.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <initializer_list>
#include <cstdint>
#include <tuple>
#include <type_traits>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/fwikkt.h"
#include "fwi_kernels.cuh"

namespace fwi {

struct Err {
  int code;
  std::string msg;
};

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw Err{FWI_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};           \
  } while (0)
// Kernel profile (diagnostics, fwi_kernel_profile): while enabled, every
// kernel launched directly (not inside a stream capture) is preceded by
// KPROF(name, level, bytes, stream), which records a CUDA event on the stream,
// and followed by KCHECK(), which records a second one.  Per (kernel, level)
// the profile sums launches, event time and the algorithmic bytes the launch
// site states (each operand and result counted once); the time between one
// launch's end event and the next launch's start event is summed as gap time.
struct ProfRow {
  long long n = 0;
  double ms = 0.0, bytes = 0.0;
};
struct Prof {
  bool on = false;
  bool pending = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev;                         // 2 per recorded launch
  std::vector<std::pair<std::string, int>> key;        // per recorded launch
  std::vector<double> bytes;
  size_t used = 0;
  std::map<std::pair<std::string, int>, ProfRow> rows;
  double gap_ms = 0.0;
  long long gaps = 0;
  void harvest() {
    for (size_t k = 0; k < used; ++k) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]) == cudaSuccess) {
        ProfRow &r = rows[key[k]];
        r.n += 1;
        r.ms += ms;
        r.bytes += bytes[k];
      }
      if (k > 0 && cudaEventElapsedTime(&ms, ev[2 * k - 1], ev[2 * k]) == cudaSuccess) {
        gap_ms += ms;
        ++gaps;
      }
    }
    used = 0;
  }
  void clear() {
    rows.clear();
    gap_ms = 0.0;
    gaps = 0;
    used = 0;
    pending = false;
  }
};
static Prof g_prof;

static void prof_begin(const char *name, int level, double nbytes, cudaStream_t s) {
  Prof &P = g_prof;
  P.pending = false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  if (P.used >= 8192) {
    if (cudaStreamSynchronize(s) != cudaSuccess) return;
    P.harvest();
  }
  while (P.ev.size() < 2 * (P.used + 1)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    P.ev.push_back(e);
  }
  if (P.key.size() <= P.used) { P.key.resize(P.used + 1); P.bytes.resize(P.used + 1); }
  P.key[P.used] = {name, level};
  P.bytes[P.used] = nbytes;
  P.st = s;
  if (cudaEventRecord(P.ev[2 * P.used], s) != cudaSuccess) return;
  P.pending = true;
}
static void prof_end() {
  Prof &P = g_prof;
  if (!P.pending) return;
  P.pending = false;
  if (cudaEventRecord(P.ev[2 * P.used + 1], P.st) == cudaSuccess) ++P.used;
}
#define KPROF(name, level, nbytes, stream)                                      \
  do {                                                                          \
    if (::fwi::g_prof.on) ::fwi::prof_begin(name, level, (double)(nbytes), stream); \
  } while (0)

// Every kernel launch of the library is followed by KCHECK(), which also
// counts it (graph replays add the number of kernels captured in the graph)
// and closes its profile record.
static std::atomic<unsigned long long> g_launches{0};
#define KCHECK()                     \
  do {                               \
    ::fwi::g_launches.fetch_add(1);  \
    CK(cudaGetLastError());          \
    if (::fwi::g_prof.pending) ::fwi::prof_end(); \
  } while (0)

static void fail(int code, const std::string &m) { throw Err{code, m}; }

// Every cudaMalloc / cudaMallocHost / cudaFree / cudaFreeHost the library makes
// (diagnostics: fwi_memory_calls).
static std::atomic<unsigned long long> g_memcalls{0};

// Every pointer starts on a 16-byte boundary (vector-access kernel variants).
static inline bool aligned16(std::initializer_list<const void *> ps) {
  for (const void *p : ps)
    if (reinterpret_cast<uintptr_t>(p) & 15u) return false;
  return true;
}

template <typename T> struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void release() {
    if (p) { cudaFree(p); g_memcalls.fetch_add(1); }
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    if (count == n && p) return;
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc((void **)&p, count * sizeof(T));
    g_memcalls.fetch_add(1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      fail(FWI_E_NOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    n = count;
  }
  void upload(const std::vector<T> &h, cudaStream_t s) {
    alloc(h.size());
    if (!h.empty()) CK(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void zero(cudaStream_t s) {
    if (n) CK(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
};

static int grid_for(long long n, int threads, int cap = 4096) {
  long long g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// --------------------------------------------------------------------------
// problem description
// --------------------------------------------------------------------------
struct Instance {
  fwi_grid g{};
  int Nx = 0, Nz = 0;
  std::vector<double> freqs;
  int n_src = 0;
  std::vector<int> src_ix, src_iz, rec_off, rec_ix, rec_iz;
  std::vector<double> src_amp, rec_w;
  bool has_survey = false, has_model = false, has_data = false;
  double gamma_ref = 0.0;
  DBuf<double> layer;   // padded gamma with the frozen layer [Nz*Nx]
  DBuf<double> s;       // core model [nz*nx]
  DBuf<double2> d;      // observed data [n_freq * rec_total]
  int blk0 = 0;
  int nlev = 1;
  long long ctrl = 0;
  int rec_total() const { return rec_off.empty() ? 0 : rec_off.back(); }
};

struct LevelTables {
  std::vector<BlkDev> hM, hA;
  std::vector<TileDev> htiles;
  std::vector<StripDev> hstrips, hstrips2, hrstrips, hpstrips;
  std::vector<int> ht0, ht1, hs0, hs1;
  DBuf<BlkDev> blksM, blksA;
  DBuf<TileDev> tiles;
  DBuf<StripDev> strips, strips2, rstrips;   // rstrips: coarse-column strips of the restriction to l + 1
  DBuf<StripDev> pstrips;                    // coarse-column strips of the prolongation from l + 1
  DBuf<int> t0, t1, s0, s1;   // per block: its row tiles [t0, t1), its column strips [s0, s1)
  long long field = 0;  // complex elements of one field on this level
  int n_tiles = 0;
  int n_strips = 0;
  int n_strips2 = 0;
  int n_rstrips = 0;
  int n_pstrips = 0;
};

template <typename T> struct Work {
  typedef typename cplx<T>::t T2;
  int ready = 0;
  // multigrid fields per global level (index 0 unused for b, x)
  DBuf<T2> lx[MAX_LEVELS], lb[MAX_LEVELS], lt[MAX_LEVELS];
  DBuf<T2> t0a, t0b;                                   // level-0 smoother buffers
  DBuf<T2> r, rh, p, p2, v, s, t, ph, sh;              // BiCGStab (p2: ping-pong partner of p)
  DBuf<BiState> bst;
  DBuf<int> done;                                      // per-block "finished" flags of the inner solve
  DBuf<T2> u;                                          // forward wavefields (precision T)
  // FGMRES
  int m = 0;
  long long n = 0;
  long long ld = 0;    // basis stride: n rounded up to 64 elements (256-byte aligned vectors)
  DBuf<T> V, Z, vin, zout, tmp, rhs, sol;              // basis, staging, sweep rhs/solution
  DBuf<T *> dptrV, dptrZ;
  DBuf<double> H, cs, sn, g, hcol, hsum, y, scal, partial_flat;
  // preconditioner graph
  cudaGraphExec_t graph = nullptr;
  std::string graph_key;
  unsigned long long graph_kernels = 0;
  // device-controlled FGMRES restart cycle: WHILE node over Arnoldi steps
  cudaGraphExec_t cyc = nullptr;
  std::string cyc_key;
  unsigned long long cyc_body_kernels = 0, cyc_tail_kernels = 0;
  DBuf<FgCtl> ctl;
  DBuf<T> wst;                                         // staging of the new Arnoldi vector
  DBuf<T> ob[8];                                       // outer BiCGStab: r, rh, p, v, s, t, ph, sh
  ~Work() {
    if (graph) cudaGraphExecDestroy(graph);
    if (cyc) cudaGraphExecDestroy(cyc);
  }
};

struct Ctx {
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<Instance> inst;
  // block layout
  bool layout_ok = false;
  int B = 0;
  std::vector<long long> blk_off;  // level 0
  std::vector<int> blk_inst, blk_freq, blk_src, blk_Nx;
  long long F0 = 0, Nc = 0, nkkt = 0;
  DBuf<long long> d_blk_off;
  DBuf<int> d_blk_Nx;
  DBuf<InstDev> d_inst;
  std::vector<InstDev> h_inst;
  // receivers (level 0 field indices)
  std::vector<long long> rec_node;                 // per survey receiver entry (all blocks)
  std::vector<double> rec_w;
  std::vector<long long> rec_data;                 // index into per-instance data arrays
  DBuf<long long> d_rec_node, d_unode, d_F_node;
  DBuf<double> d_rec_w, d_F_w2;
  DBuf<int> d_uoff, d_uidx;
  int n_unique = 0, n_F = 0;
  DBuf<long long> d_src_node;
  DBuf<double2> d_src_amp;
  // hierarchy
  int model_version = 1;
  std::string hier_key;
  int ls = 1, nlev_max = 1;
  int ls_p[2] = {1, 1};   // first shared-memory level for complex64 / complex128
  const int *cur_skip = nullptr;   // set inside an inner solve: per-block finished flags
  LevelTables lv[MAX_LEVELS];
  std::vector<OpDev> h_ops;
  DBuf<OpDev> d_ops;
  DBuf<double2> st64;
  DBuf<float2> st32;
  DBuf<double> gam64;
  DBuf<float> gam32;
  DBuf<double2> inv;
  DBuf<long long> inv_off;
  DBuf<double2> dg64, dgi64;
  DBuf<float2> dg32, dgi32;
  DBuf<int> d_inst_nlev;
  DBuf<double> cfK, cfG;   // per-block coupling factors (KKT scaled, gradient)
  // ILU(0) factors of every A operator ([5][total] complex: 1/d, lw, ln, ce, cs)
  std::string ilu_key;
  DBuf<double2> ilu64;
  DBuf<float2> ilu32;
  DBuf<long long> ilu_off;  // per operator id: offset of its factors (-1: none)
  long long ilu_stride = 0;
  int ilu_maxnz = 0;
  size_t smem_bytes[2] = {0, 0};
  // forward state
  bool have_fwd = false;
  bool u64_valid = false;          // u64 holds converged wavefields of the current layout
  int fwd_version = 0;
  DBuf<double2> u64, f64, rho64, e64;
  DBuf<double2> q, r;                         // predicted data, residual per receiver entry
  std::vector<double> misfit;
  // KKT FP64 state
  DBuf<double> b64, xi64, rho_k64, tmp64;
  DBuf<SegDev> d_segs;
  std::vector<SegDev> h_segs;
  DBuf<double> seg_partial, inst_norm2, inst_fac;
  DBuf<int> d_flag;
  DBuf<double2> partial;   // per-tile partial sums [n_tiles0 * 3]
  DBuf<double2> partial_s; // per-strip partial sums [n_strips0 * 3]
  DBuf<double> blkfac, blkn0, blkn;   // per-block factors / norms
  DBuf<double> misfit_d, inst_gref;
  int u_version32 = -1, u_version64 = -1;
  Work<float> w32;
  Work<double> w64;
  // quasi-Newton H block of the preconditioner (opts.hblock = 1): m pairs of
  // the scaled control, S and Y as [m][Nc]; the folded 2m x 2m matrix of the
  // compact form for the eps in qn_eps
  int qn_m = 0, qn_version = 0;
  double qn_eps = 0.0;
  DBuf<double> qnS, qnY, qnMf, qnPart;
  std::vector<double> qn_SY, qn_YY;
  double *pin = nullptr;  // pinned scalars
  int *pinflag = nullptr;
  // live timing of the level-0 stencil kernel (k_field_op): event pairs around
  // direct launches on this context's stream, with the launch's algorithmic bytes
  int timer_on = 0;
  bool timer_blocked = false;      // set by calls that must not allocate (no timed launches)
  int dev = -1;                    // CUDA device of the context (recorded at first device use)
  std::vector<cudaEvent_t> ev_a, ev_b;
  std::vector<double> ev_bytes;    // algorithmic bytes per processed node of each timed launch
  std::vector<double> ev_pbytes;   // bytes per processed node of the fused pass itself
  DBuf<unsigned long long> ev_work; // nodes processed by each timed launch (device counters)
  size_t ev_used = 0;
  double timer_ms = 0.0, timer_bytes = 0.0, timer_pbytes = 0.0;
  long long timer_n = 0;
  void harvest() {
    std::vector<unsigned long long> work(ev_used, 0);
    if (ev_used) {
      cudaMemcpy(work.data(), ev_work.p, ev_used * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
      cudaMemset(ev_work.p, 0, ev_used * sizeof(unsigned long long));
    }
    for (size_t q = 0; q < ev_used; ++q) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_a[q], ev_b[q]) == cudaSuccess) {
        timer_ms += ms;
        timer_bytes += ev_bytes[q] * (double)work[q];
        timer_pbytes += ev_pbytes[q] * (double)work[q];
        ++timer_n;
      }
    }
    ev_used = 0;
  }

  bool own_stream = false;
  ~Ctx() {
    for (auto e : ev_a) cudaEventDestroy(e);
    for (auto e : ev_b) cudaEventDestroy(e);
    if (pin) { cudaFreeHost(pin); g_memcalls.fetch_add(1); }
    if (pinflag) { cudaFreeHost(pinflag); g_memcalls.fetch_add(1); }
    if (own_stream && st) cudaStreamDestroy(st);
  }

  // core nodes x blocks summed over the instances (the coupling reduction's work)
  long long cpl_nodes() const {
    long long t = 0;
    for (size_t i = 0; i < inst.size() && i < h_inst.size(); ++i)
      t += (long long)inst[i].g.nx * inst[i].g.nz * (h_inst[i].blk1 - h_inst[i].blk0);
    return t;
  }
  template <typename T> Work<T> &work();
  template <typename T> LevelView<T> viewA();
  template <typename T> LevelView<T> viewM(int l);

  // ------------------------------------------------------------------------
  void build_layout();
  void build_hierarchy(const fwi_opts &o);
  template <typename T> void ensure_work(const fwi_opts &o);
  template <typename T> void ensure_krylov(const fwi_opts &o);
  template <typename T> void launch_coarse(const CoarseArgs &ca, size_t smem, const typename cplx<T>::t *b,
                                           typename cplx<T>::t *x, int cj, int nthreads);
  template <typename T> const typename cplx<T>::t *u_T();
  int gradient(const fwi_opts &o, double *misfit_out, double *grad, int on_device, fwi_stats *stats);
  int newton_step(const fwi_opts &o, double *ds, int on_device, fwi_stats *stats);
  int rsgn_solve(const fwi_opts &o, fwi_stats *stats);
  int normal_lambda_max(const fwi_opts &o, int iters, double *lambda, fwi_stats *stats);
  int rsgn_step(const fwi_opts &o, double *ds, int on_device, fwi_stats *stats);
  int hessian_apply(const fwi_opts &o, const double *v, double *hv, int on_device, fwi_stats *stats);
  void hblock_set(int m, const double *S, const double *Y, int on_device);
  void hblock_prepare(const fwi_opts &o);
  template <typename T> void hblock_apply(T *zs, const fwi_opts &o);
  int qn_grid() const { return (int)std::max(1LL, std::min((long long)FLAT_BLOCKS, (Nc + FLAT_THREADS - 1) / FLAT_THREADS)); }
  int hb_key(const fwi_opts &o) const { return (o.hblock && qn_m > 0) ? qn_version : 0; }
  void apply_update(double *ds, int on_device);
  void write_ctrl(const double *src_ctrl_dev, double *dst, int on_device, const double *fac);
  template <typename T> void mg_cycle(const typename cplx<T>::t *b, typename cplx<T>::t *x, int cj,
                                      const fwi_opts &o, const BFuse<T> *fz = nullptr);
  template <typename T> void bicg_update_into(const BFuse<T> &fz);
  void ensure_ilu();
  template <typename T> void ilu_apply(int cj, const typename cplx<T>::t *b, typename cplx<T>::t *x);
  template <typename T> void inner_solve(const typename cplx<T>::t *b, typename cplx<T>::t *x, int cj,
                                         int iters, double tol, const fwi_opts &o, long long *count,
                                         bool ilu = false);
  template <typename T> void mg_cycle_into(const typename cplx<T>::t *b, typename cplx<T>::t *x, int cj,
                                           const fwi_opts &o, typename cplx<T>::t *const *lx,
                                           typename cplx<T>::t *const *lb, typename cplx<T>::t *const *lt,
                                           typename cplx<T>::t *t0);
  template <typename T> bool timer_begin(int level, LevelView<T> &L);
  template <typename T> void smooth(int nu, bool zero, int cj, T wj, const typename cplx<T>::t *bl,
                                    typename cplx<T>::t *&cur, typename cplx<T>::t *&oth, int l,
                                    const BFuse<T> *fz = nullptr);
  template <typename T> void resid_restrict(int cj, int l, const typename cplx<T>::t *x, const typename cplx<T>::t *b,
                                            typename cplx<T>::t *bc);
  template <typename T> void prolong(int l, const LevelView<T> &Lf, const LevelView<T> &Lc,
                                     const typename cplx<T>::t *xc, typename cplx<T>::t *xf);
  void timer_end(int streams, int pass_streams, size_t elem_bytes);
  template <typename T> void apply_dots(int cj, const typename cplx<T>::t *x, typename cplx<T>::t *y,
                                        const typename cplx<T>::t *a, int nd);
  template <typename T> void jacobi2(int cj, T wj, const typename cplx<T>::t *x, const typename cplx<T>::t *b,
                                     typename cplx<T>::t *y, int level, const BFuse<T> *fz = nullptr);
  template <typename T> void field_op(int mode, int cj, T w, const typename cplx<T>::t *x,
                                      const typename cplx<T>::t *b, typename cplx<T>::t *y, bool opA,
                                      int level);
  template <typename T> void block_dots(int nd, const typename cplx<T>::t *a0, const typename cplx<T>::t *b0,
                                        const typename cplx<T>::t *a1, const typename cplx<T>::t *b1,
                                        const typename cplx<T>::t *a2, const typename cplx<T>::t *b2);
  template <typename T> void kkt_matvec(const T *xi, T *y, double eps, const typename cplx<T>::t *u);
  template <typename T> void precond(const T *v, T *z, const fwi_opts &o, long long *count,
                                     const typename cplx<T>::t *u);
  template <typename T> void precond_any(const T *v, T *z, const fwi_opts &o, long long *count,
                                         const typename cplx<T>::t *u);
  template <typename T> int fgmres(const T *rhs, T *x, double tol, int maxit, double eps, const fwi_opts &o,
                                   int *iters, long long *inner, const typename cplx<T>::t *u);
  template <typename T> void multidot(long long n, int nv, T *const *dV, const T *w, double *out, int acc,
                                      int pm);
  template <typename T> void multi_axpy(long long n, int nv, T *const *dV, const double *coef, double sign, T *w);
  template <typename T> void fgmres_cycle_graph(const fwi_opts &o, double eps, T *x, const typename cplx<T>::t *u);
  template <typename T> int bicgstab_outer(const T *rhs, T *x, double tol, int maxit, double eps, const fwi_opts &o,
                                           int *iters, long long *inner, const typename cplx<T>::t *u);
  double orth_loss = 0.0;   // max |I - V^T V| of the FGMRES bases of the last KKT solve (check_orth)
  void forward(const fwi_opts &o, fwi_stats *stats);
  template <typename T> int refined_solve(const double2 *rhs, double2 *x, int cj, const fwi_opts &o,
                                          fwi_stats *stats, bool warm = false);
  void seg_norms(const double *x);
  int kkt_solve(const fwi_opts &o, fwi_stats *stats);
  void sync() {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) fail(FWI_E_CUDA, "internal: stream synchronisation during a capture");
    CK(cudaStreamSynchronize(st));
    if (ev_used) harvest();
    if (g_prof.used) g_prof.harvest();
  }
};

template <> Work<float> &Ctx::work<float>() { return w32; }
template <> Work<double> &Ctx::work<double>() { return w64; }

template <typename T> static const typename cplx<T>::t *st_ptr(Ctx &c);
template <> const float2 *st_ptr<float>(Ctx &c) { return c.st32.p; }
template <> const double2 *st_ptr<double>(Ctx &c) { return c.st64.p; }
template <typename T> static const typename cplx<T>::t *dg_ptr(Ctx &c);
template <> const float2 *dg_ptr<float>(Ctx &c) { return c.dg32.p; }
template <> const double2 *dg_ptr<double>(Ctx &c) { return c.dg64.p; }
template <typename T> static const typename cplx<T>::t *dgi_ptr(Ctx &c);
template <> const float2 *dgi_ptr<float>(Ctx &c) { return c.dgi32.p; }
template <> const double2 *dgi_ptr<double>(Ctx &c) { return c.dgi64.p; }
template <typename T> static const T *gam_ptr(Ctx &c);
template <> const float *gam_ptr<float>(Ctx &c) { return c.gam32.p; }
template <> const double *gam_ptr<double>(Ctx &c) { return c.gam64.p; }

template <typename T>
void Ctx::launch_coarse(const CoarseArgs &ca, size_t smem, const typename cplx<T>::t *b, typename cplx<T>::t *x,
                        int cj, int nthreads) {
  KPROF("k_coarse_cycle", ca.ls, 2.0 * sizeof(typename cplx<T>::t) * lv[ca.ls].field, st);
  if (nthreads == 1024) {
    if (cj) k_coarse_cycle<T, true, 1024><<<B, 1024, smem, st>>>(ca, st_ptr<T>(*this), dgi_ptr<T>(*this), b, x);
    else k_coarse_cycle<T, false, 1024><<<B, 1024, smem, st>>>(ca, st_ptr<T>(*this), dgi_ptr<T>(*this), b, x);
  } else {
    if (cj) k_coarse_cycle<T, true, 512><<<B, 512, smem, st>>>(ca, st_ptr<T>(*this), dgi_ptr<T>(*this), b, x);
    else k_coarse_cycle<T, false, 512><<<B, 512, smem, st>>>(ca, st_ptr<T>(*this), dgi_ptr<T>(*this), b, x);
  }
  KCHECK();
}

template <typename T> LevelView<T> Ctx::viewA() {
  LevelView<T> v;
  v.ops = d_ops.p; v.blks = lv[0].blksA.p; v.tiles = lv[0].tiles.p;
  v.st = st_ptr<T>(*this); v.gam = gam_ptr<T>(*this);
  v.dg = dg_ptr<T>(*this); v.dgi = dgi_ptr<T>(*this);
  v.skip = cur_skip;
  v.work = nullptr;
  v.n_tiles = lv[0].n_tiles; v.n_blocks = B;
  v.strips = lv[0].strips.p; v.n_strips = lv[0].n_strips;
  v.strips2 = lv[0].strips2.p; v.n_strips2 = lv[0].n_strips2;
  return v;
}
template <typename T> LevelView<T> Ctx::viewM(int l) {
  LevelView<T> v;
  v.ops = d_ops.p; v.blks = lv[l].blksM.p; v.tiles = lv[l].tiles.p;
  v.st = st_ptr<T>(*this); v.gam = gam_ptr<T>(*this);
  v.dg = dg_ptr<T>(*this); v.dgi = dgi_ptr<T>(*this);
  v.skip = cur_skip;
  v.work = nullptr;
  v.n_tiles = lv[l].n_tiles; v.n_blocks = B;
  v.strips = lv[l].strips.p; v.n_strips = lv[l].n_strips;
  v.strips2 = lv[l].strips2.p; v.n_strips2 = lv[l].n_strips2;
  return v;
}

// --------------------------------------------------------------------------
// layout of the batch (blocks, receivers, sources)
// --------------------------------------------------------------------------
static int auto_levels(int Nx, int Nz, int max_nodes = 256, int min_dim = 3) {
  int L = 1, nx = Nx, nz = Nz;
  while ((long long)nx * nz > max_nodes && nx / 2 >= min_dim && nz / 2 >= min_dim) {
    nx /= 2; nz /= 2; ++L;
  }
  return L;
}

void Ctx::build_layout() {
  if (layout_ok) return;
  if (dev < 0) CK(cudaGetDevice(&dev));
  if (!st) {
    // the legacy default stream cannot be captured into a CUDA graph: use a
    // private blocking stream (it still orders with the legacy default stream)
    CK(cudaStreamCreate(&st));
    own_stream = true;
  }
  for (size_t i = 0; i < inst.size(); ++i)
    if (!inst[i].has_survey || !inst[i].has_model) fail(FWI_E_INVAL, "every instance needs a survey and a model");
  B = 0; F0 = 0; Nc = 0;
  blk_off.clear(); blk_inst.clear(); blk_freq.clear(); blk_src.clear(); blk_Nx.clear();
  h_inst.clear();
  for (size_t i = 0; i < inst.size(); ++i) {
    Instance &I = inst[i];
    I.blk0 = B;
    I.ctrl = Nc;
    InstDev d;
    d.npml = I.g.npml; d.nx = I.g.nx; d.nz = I.g.nz;
    d.blk0 = B;
    for (size_t f = 0; f < I.freqs.size(); ++f)
      for (int k = 0; k < I.n_src; ++k) {
        blk_off.push_back(F0);
        blk_inst.push_back((int)i); blk_freq.push_back((int)f); blk_src.push_back(k);
        blk_Nx.push_back(I.Nx);
        F0 += (long long)I.Nx * I.Nz;
        ++B;
      }
    d.blk1 = B;
    d.ctrl = Nc;
    Nc += (long long)I.g.nx * I.g.nz;
    h_inst.push_back(d);
  }
  nkkt = 4 * F0 + Nc;
  d_inst.upload(h_inst, st);
  d_blk_off.upload(blk_off, st);
  d_blk_Nx.upload(blk_Nx, st);
  // receivers: one entry per (block, survey receiver of its source)
  rec_node.clear(); rec_w.clear(); rec_data.clear();
  std::vector<long long> src_node;
  std::vector<double2> amp;
  for (int b = 0; b < B; ++b) {
    Instance &I = inst[blk_inst[b]];
    int k = blk_src[b], f = blk_freq[b];
    int p = I.g.npml;
    src_node.push_back(blk_off[b] + (long long)(I.src_iz[k] + p) * I.Nx + (I.src_ix[k] + p));
    amp.push_back(make_double2(I.src_amp[2 * k], I.src_amp[2 * k + 1]));
    for (int e = I.rec_off[k]; e < I.rec_off[k + 1]; ++e) {
      rec_node.push_back(blk_off[b] + (long long)(I.rec_iz[e] + p) * I.Nx + (I.rec_ix[e] + p));
      rec_w.push_back(I.rec_w[e]);
      rec_data.push_back((long long)f * I.rec_total() + e);
    }
  }
  d_src_node.upload(src_node, st);
  d_src_amp.upload(amp, st);
  d_rec_node.upload(rec_node, st);
  d_rec_w.upload(rec_w, st);
  // unique receiver nodes (for the scatter Q^T W^T W r and the diagonal F)
  std::vector<int> order(rec_node.size());
  for (size_t q = 0; q < order.size(); ++q) order[q] = (int)q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return rec_node[a] < rec_node[b]; });
  std::vector<long long> unode;
  std::vector<int> uoff, uidx;
  std::vector<double> fw2;
  for (size_t q = 0; q < order.size(); ++q) {
    if (q == 0 || rec_node[order[q]] != rec_node[order[q - 1]]) {
      unode.push_back(rec_node[order[q]]);
      uoff.push_back((int)q);
      fw2.push_back(0.0);
    }
    uidx.push_back(order[q]);
    fw2.back() += rec_w[order[q]] * rec_w[order[q]];
  }
  uoff.push_back((int)order.size());
  n_unique = (int)unode.size();
  n_F = n_unique;
  d_unode.upload(unode, st);
  d_uoff.upload(uoff, st);
  d_uidx.upload(uidx, st);
  d_F_node.upload(unode, st);
  d_F_w2.upload(fw2, st);
  // segments of packed vectors: [du | lm | ds], one per instance and region
  h_segs.clear();
  for (size_t i = 0; i < inst.size(); ++i) {
    long long b0 = blk_off[h_inst[i].blk0];
    long long b1 = h_inst[i].blk1 < B ? blk_off[h_inst[i].blk1] : F0;
    h_segs.push_back(SegDev{2 * b0, 2 * b1, (int)i});
    h_segs.push_back(SegDev{2 * F0 + 2 * b0, 2 * F0 + 2 * b1, (int)i});
    h_segs.push_back(SegDev{4 * F0 + h_inst[i].ctrl, 4 * F0 + h_inst[i].ctrl + (long long)inst[i].g.nx * inst[i].g.nz, (int)i});
  }
  d_segs.upload(h_segs, st);
  seg_partial.alloc(h_segs.size() * 64);
  inst_norm2.alloc(inst.size());
  inst_fac.alloc(inst.size());
  d_flag.alloc(1);
  if (!pin) {
    CK(cudaMallocHost((void **)&pin, 64 * sizeof(double)));
    CK(cudaMallocHost((void **)&pinflag, 4 * sizeof(int)));
    g_memcalls.fetch_add(2);
  }
  layout_ok = true;
  u64_valid = false;
  hier_key.clear();
  w32.ready = 0;
  w64.ready = 0;
}

// --------------------------------------------------------------------------
// a1: per-frequency set-up -- stretch arrays, gamma on every level, operator
// tables, coarsest dense inverses (FP64)
// --------------------------------------------------------------------------
// Key of the multigrid hierarchy and launch tables built for these options
// and the current models.
static std::string hierarchy_key(int model_version, const fwi_opts &o) {
  char key[256];
  snprintf(key, sizeof key, "%d|%d|%.17g|%.17g|%d", model_version, o.mg_levels, o.shift_beta, o.sigma_cap,
           o.strip_rows);
  return key;
}

void Ctx::build_hierarchy(const fwi_opts &o) {
  build_layout();
  const std::string key = hierarchy_key(model_version, o);
  if (hier_key == key) return;
  const int srows = o.strip_rows;
  const int n_inst = (int)inst.size();
  // levels per instance
  nlev_max = 1;
  for (auto &I : inst) {
    int L = auto_levels(I.Nx, I.Nz);
    if (o.mg_levels > 0) L = std::min(L, o.mg_levels);
    if (L > MAX_LEVELS) L = MAX_LEVELS;
    I.nlev = L;
    nlev_max = std::max(nlev_max, L);
  }
  // level dims per instance
  auto dims = [&](const Instance &I, int l, int &nx, int &nz) {
    nx = I.Nx; nz = I.Nz;
    for (int q = 0; q < l; ++q) { nx /= 2; nz /= 2; }
  };
  // shared-memory start level: the first level from which every instance's
  // remaining levels (3 vectors and the operator data each) fit in the per-CTA
  // budget (c64);
  // complex128 may need a coarser start.
  const size_t budget = 220 * 1024;
  auto smem_from = [&](int l0, size_t elem) {
    size_t mx = 0;
    for (auto &I : inst) {
      size_t s = 0;
      for (int l = l0; l < I.nlev; ++l) { int nx, nz; dims(I, l, nx, nz); s += smem_level_bytes(nx, nz, elem); }
      mx = std::max(mx, s);
    }
    return mx;
  };
  int minlev = nlev_max;
  for (auto &I : inst) minlev = std::min(minlev, I.nlev);
  for (int p = 0; p < 2; ++p) {
    size_t elem = p ? sizeof(double2) : sizeof(float2);
    int l0 = 1;
    while (l0 < minlev - 1 && smem_from(l0, elem) > budget) ++l0;
    if (minlev < 2) l0 = 0;  // single-level instances: the whole cycle is the coarse solve
    ls_p[p] = l0;
    smem_bytes[p] = smem_from(l0, elem);
  }
  ls = std::max(ls_p[0], ls_p[1]);   // tiles and global level tables are built up to here
  if (smem_bytes[1] > 227 * 1024 || smem_bytes[0] > 227 * 1024)
    fail(FWI_E_INVAL, "grids too different for one batch (coarse levels exceed shared memory)");
  // operators
  h_ops.clear();
  std::vector<AxisDev> axes;
  long long st_tot = 0, dg_tot = 0;
  std::vector<long long> gam_off(n_inst * MAX_LEVELS, -1);
  long long gam_tot = 0;
  for (int i = 0; i < n_inst; ++i)
    for (int l = 0; l < inst[i].nlev; ++l) {
      int nx, nz; dims(inst[i], l, nx, nz);
      gam_off[i * MAX_LEVELS + l] = gam_tot;
      gam_tot += (long long)nx * nz;
    }
  // op ids: A ops [inst][freq], M ops [inst][freq][level]
  std::vector<int> opA(B), opM0(B);
  std::vector<std::vector<int>> opM(MAX_LEVELS, std::vector<int>(B, -1));
  std::vector<int> coarse_ops;
  std::map<std::pair<int, int>, int> aid;
  std::map<std::tuple<int, int, int>, int> mid;
  for (int i = 0; i < n_inst; ++i) {
    Instance &I = inst[i];
    double L = I.g.npml * I.g.h;
    double smax = I.g.npml > 0 ? 3.0 * I.g.pml_c * std::log(1.0 / I.g.pml_R) / (2.0 * L) : 0.0;
    for (size_t f = 0; f < I.freqs.size(); ++f) {
      double om = 2.0 * M_PI * I.freqs[f];
      for (int kind = 0; kind < 2; ++kind) {
        int nl = kind == 0 ? 1 : I.nlev;
        for (int l = 0; l < nl; ++l) {
          int nx, nz; dims(I, l, nx, nz);
          double hl = I.g.h, x0 = 0.0;
          for (int q = 0; q < l; ++q) { x0 += hl; hl *= 2.0; }
          OpDev od;
          od.nx = nx; od.nz = nz;
          od.st = st_tot;
          od.gam = gam_off[i * MAX_LEVELS + l];
          od.dg = dg_tot;
          dg_tot += (long long)nx * nz;
          double beta = kind == 0 ? 0.0 : o.shift_beta;
          od.mass_re = (om * hl) * (om * hl);
          od.mass_im = beta * (om * hl) * (om * hl);
          AxisDev ad;
          ad.dst = st_tot; ad.nx = nx; ad.nz = nz; ad.x0 = x0; ad.z0 = x0; ad.hl = hl;
          ad.xlo = I.g.npml * I.g.h; ad.xhi = (I.g.npml + I.g.nx - 1) * I.g.h;
          ad.zlo = I.g.npml * I.g.h; ad.zhi = (I.g.npml + I.g.nz - 1) * I.g.h;
          ad.L = L; ad.smax = smax; ad.omega = om; ad.cap = kind == 0 ? -1.0 : o.sigma_cap;
          axes.push_back(ad);
          st_tot += 2 * nx + 2 * nz + 2;
          int id = (int)h_ops.size();
          h_ops.push_back(od);
          if (kind == 0) aid[{i, (int)f}] = id;
          else {
            mid[{i, (int)f, l}] = id;
            if (l == I.nlev - 1) coarse_ops.push_back(id);
          }
        }
      }
    }
  }
  d_ops.upload(h_ops, st);
  std::vector<AxisDev> hax = axes;
  DBuf<AxisDev> dax;
  dax.upload(hax, st);
  st64.alloc(st_tot);
  st32.alloc(st_tot);
  KPROF("k_stretch_setup", -1, 0, st);
  k_stretch_setup<<<(int)axes.size(), 128, 0, st>>>(dax.p, (int)axes.size(), st64.p, st32.p);
  KCHECK();
  // gamma on every level
  gam64.alloc(gam_tot);
  gam32.alloc(gam_tot);
  for (int i = 0; i < n_inst; ++i) {
    Instance &I = inst[i];
    long long n0 = (long long)I.Nx * I.Nz;
    KPROF("k_gamma_fill", -1, 0, st);
    k_gamma_fill<<<grid_for(n0, 256), 256, 0, st>>>(I.layer.p, I.s.p, I.Nx, I.Nz, I.g.npml, I.g.nx, I.g.nz,
                                                     gam64.p + gam_off[i * MAX_LEVELS], gam32.p + gam_off[i * MAX_LEVELS]);
    KCHECK();
    for (int l = 1; l < I.nlev; ++l) {
      int nxf, nzf, nxc, nzc;
      dims(I, l - 1, nxf, nzf); dims(I, l, nxc, nzc);
      KPROF("k_gamma_restrict", -1, 0, st);
      k_gamma_restrict<<<grid_for((long long)nxc * nzc, 256), 256, 0, st>>>(
          gam64.p + gam_off[i * MAX_LEVELS + l - 1], nxf, nzf, nxc, nzc, gam64.p + gam_off[i * MAX_LEVELS + l],
          gam32.p + gam_off[i * MAX_LEVELS + l]);
      KCHECK();
    }
  }
  // diagonal of every operator and its inverse
  dg64.alloc(dg_tot); dgi64.alloc(dg_tot); dg32.alloc(dg_tot); dgi32.alloc(dg_tot);
  KPROF("k_diag_setup", -1, 0, st);
  k_diag_setup<<<(int)h_ops.size(), 256, 0, st>>>(d_ops.p, st64.p, gam64.p, dg64.p, dgi64.p, dg32.p, dgi32.p);
  KCHECK();
  // coarsest inverses
  std::vector<long long> h_inv_off(h_ops.size(), -1), aug_off, inv_off_l;
  std::vector<int> cdims;
  long long inv_tot = 0, aug_tot = 0;
  for (int id : coarse_ops) {
    long long n = (long long)h_ops[id].nx * h_ops[id].nz;
    h_inv_off[id] = inv_tot;
    inv_off_l.push_back(inv_tot);
    aug_off.push_back(aug_tot);
    cdims.push_back((int)n);
    inv_tot += n * n;
    aug_tot += n * 2 * n;
  }
  inv.alloc(inv_tot);
  inv_off.upload(h_inv_off, st);
  {
    DBuf<double2> aug;
    aug.alloc(aug_tot);
    DBuf<int> dids, ddims, dstat;
    DBuf<long long> daoff, dioff;
    dids.upload(coarse_ops, st);
    ddims.upload(cdims, st);
    daoff.upload(aug_off, st);
    dioff.upload(inv_off_l, st);
    dstat.alloc(1);
    dstat.zero(st);
    KPROF("k_coarse_assemble", -1, 0, st);
    k_coarse_assemble<<<(int)coarse_ops.size(), 256, 0, st>>>(d_ops.p, dids.p, daoff.p, st64.p, gam64.p, aug.p);
    KCHECK();
    KPROF("k_gauss_jordan", -1, 0, st);
    k_gauss_jordan<<<(int)coarse_ops.size(), 256, 0, st>>>(ddims.p, daoff.p, dioff.p, aug.p, inv.p, dstat.p);
    KCHECK();
    int hs = 0;
    CK(cudaMemcpyAsync(&hs, dstat.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    sync();
    if (hs) fail(FWI_E_NUMERIC, "coarsest multigrid operator is singular");
  }
  std::vector<int> hn(n_inst);
  for (int i = 0; i < n_inst; ++i) hn[i] = inst[i].nlev;
  d_inst_nlev.upload(hn, st);
  // per-level block and tile tables (all levels < nlev of each instance; the
  // smem levels need only the block tables)
  for (int l = 0; l < nlev_max; ++l) {
    LevelTables &T = lv[l];
    T.hM.assign(B, BlkDev{0, 0, 0});
    T.hA.assign(B, BlkDev{0, 0, 0});
    T.htiles.clear(); T.hstrips.clear(); T.hstrips2.clear(); T.hrstrips.clear(); T.hpstrips.clear(); T.ht0.assign(B, 0); T.ht1.assign(B, 0);
    T.hs0.assign(B, 0); T.hs1.assign(B, 0);
    long long off = 0;
    for (int b = 0; b < B; ++b) {
      int i = blk_inst[b];
      Instance &I = inst[i];
      int lq = std::min(l, I.nlev - 1);
      int nx, nz; dims(I, lq, nx, nz);
      BlkDev bd;
      bd.off = off; bd.inst = i;
      bd.op = mid[{i, blk_freq[b], lq}];
      T.hM[b] = bd;
      bd.op = aid[{i, blk_freq[b]}];
      T.hA[b] = bd;
      T.ht0[b] = (int)T.htiles.size();
      if (l <= ls)
        for (int r0 = 0; r0 < nz; r0 += TILE_ROWS) T.htiles.push_back(TileDev{b, r0});
      T.ht1[b] = (int)T.htiles.size();
      // column strips of the register-marching stencil kernel (fine levels):
      // block-major, then row band, then column, so that neighbouring strips
      // (which share halo rows and columns) run close together
      // Below level 0 the grids are 4x smaller while the work per strip is the
      // same, so the stencil strips are half as high there (twice the warps in
      // flight on an L2-resident level).
      const int sr_l = l == 0 ? srows : std::max(2, srows / 2);
      T.hs0[b] = (int)T.hstrips.size();
      if (l < std::max(ls, 1))   // level 0 always (operator apply, dots), the other global levels
        for (int r0 = 0; r0 < nz; r0 += sr_l) {
          for (int c0 = 0; c0 < nx; c0 += MARCH_COLS)
            T.hstrips.push_back(StripDev{b, c0, r0, std::min(r0 + sr_l, nz)});
          for (int c0 = 0; c0 < nx; c0 += MARCH2_COLS)
            T.hstrips2.push_back(StripDev{b, c0, r0, std::min(r0 + sr_l, nz)});
        }
      T.hs1[b] = (int)T.hstrips.size();
      if (l < ls) {
        const int ncx = nx / 2, ncz = nz / 2;   // level l + 1 (dims halve per level)
        for (int J0 = 0; J0 < ncz; J0 += RM_ROWS)
          for (int C0 = 0; C0 < ncx; C0 += RM_COLS)
            T.hrstrips.push_back(StripDev{b, C0, J0, std::min(J0 + RM_ROWS, ncz)});
        // prolongation: coarse indices J, I whose fine rows 2J, 2J + 1 and
        // columns 2I, 2I + 1 meet the fine grid (up to ncz, ncx for odd sizes)
        const int pcz = (nz + 1) / 2, pcx = (nx + 1) / 2;
        for (int J0 = 0; J0 < pcz; J0 += PM_ROWS)
          for (int C0 = 0; C0 < pcx; C0 += PM_COLS)
            T.hpstrips.push_back(StripDev{b, C0, J0, std::min(J0 + PM_ROWS, pcz)});
      }
      off += (long long)nx * nz;
    }
    T.field = off;
    T.n_tiles = (int)T.htiles.size();
    T.n_strips = (int)T.hstrips.size();
    T.strips.upload(T.hstrips, st);
    T.n_strips2 = (int)T.hstrips2.size();
    T.strips2.upload(T.hstrips2, st);
    T.n_rstrips = (int)T.hrstrips.size();
    T.rstrips.upload(T.hrstrips, st);
    T.n_pstrips = (int)T.hpstrips.size();
    T.pstrips.upload(T.hpstrips, st);
    T.blksM.upload(T.hM, st);
    T.blksA.upload(T.hA, st);
    T.tiles.upload(T.htiles, st);
    T.t0.upload(T.ht0, st);
    T.t1.upload(T.ht1, st);
    T.s0.upload(T.hs0, st);
    T.s1.upload(T.hs1, st);
  }
  partial.alloc((size_t)std::max(1, lv[0].n_tiles) * 3);
  partial_s.alloc((size_t)std::max(1, lv[0].n_strips) * 3);
  blkfac.alloc(B); blkn0.alloc(B); blkn.alloc(B);
  // coupling factors: KKT (h^2 gamma_ref omega^2) and gradient (h^2 omega^2)
  std::vector<double> cK(B), cG(B);
  for (int b = 0; b < B; ++b) {
    Instance &I = inst[blk_inst[b]];
    double om = 2.0 * M_PI * I.freqs[blk_freq[b]];
    cG[b] = I.g.h * I.g.h * om * om;
    cK[b] = cG[b] * I.gamma_ref;
  }
  cfK.upload(cK, st);
  cfG.upload(cG, st);
  sync();
  hier_key = key;
  w32.ready = 0;
  w64.ready = 0;
}

// Dynamic shared-memory limit of every instantiation of the coarse-cycle kernel.
template <typename T> static void set_coarse_smem(int bytes) {
  CK(cudaFuncSetAttribute(k_coarse_cycle<T, false, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_coarse_cycle<T, true, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_coarse_cycle<T, false, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  CK(cudaFuncSetAttribute(k_coarse_cycle<T, true, 1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
}

template <typename T> void Ctx::ensure_work(const fwi_opts &o) {
  Work<T> &w = work<T>();
  if (w.ready) return;
  for (int l = 1; l <= ls_p[sizeof(T) == 8] && l < nlev_max; ++l) {
    w.lx[l].alloc(lv[l].field); w.lb[l].alloc(lv[l].field); w.lt[l].alloc(lv[l].field);
  }
  w.t0a.alloc(F0); w.t0b.alloc(F0);
  w.r.alloc(F0); w.rh.alloc(F0); w.p.alloc(F0); w.p2.alloc(F0); w.v.alloc(F0);
  w.s.alloc(F0); w.t.alloc(F0); w.ph.alloc(F0); w.sh.alloc(F0);
  w.bst.alloc(B);
  w.done.alloc(B);
  w.u.alloc(F0);
  w.vin.alloc(nkkt); w.zout.alloc(nkkt); w.tmp.alloc(nkkt);
  w.scal.alloc(8);
  w.partial_flat.alloc((size_t)MD_CHUNK * FLAT_BLOCKS);
  if (smem_bytes[sizeof(T) == 8] > 48 * 1024) set_coarse_smem<T>((int)smem_bytes[sizeof(T) == 8]);
  if (w.graph) { cudaGraphExecDestroy(w.graph); w.graph = nullptr; }
  w.graph_key.clear();
  if (w.cyc) { cudaGraphExecDestroy(w.cyc); w.cyc = nullptr; }
  w.cyc_key.clear();
  sync();
  w.ready = 1;
  (void)o;
}

// FGMRES basis (restart m): V (m+1 vectors) and Z (m vectors) of the packed KKT size.
template <typename T> void Ctx::ensure_krylov(const fwi_opts &o) {
  ensure_work<T>(o);
  Work<T> &w = work<T>();
  int m = std::max(1, o.restart);
  if (w.m == m && w.V.p) return;
  w.m = m;
  w.n = nkkt;
  w.ld = (nkkt + 63) / 64 * 64;
  w.V.alloc((size_t)(m + 1) * w.ld);
  w.Z.alloc((size_t)m * w.ld);
  std::vector<T *> pv(m + 1), pz(m);
  for (int k = 0; k <= m; ++k) pv[k] = w.V.p + (size_t)k * w.ld;
  for (int k = 0; k < m; ++k) pz[k] = w.Z.p + (size_t)k * w.ld;
  w.dptrV.upload(pv, st);
  w.dptrZ.upload(pz, st);
  w.H.alloc((size_t)(m + 1) * m); w.cs.alloc(m); w.sn.alloc(m); w.g.alloc(m + 1);
  w.hcol.alloc(m + 1); w.hsum.alloc(m + 1); w.y.alloc(m);
  w.rhs.alloc(nkkt); w.sol.alloc(nkkt);
  w.wst.alloc(nkkt);
  w.ctl.alloc(1);
  if (w.cyc) { cudaGraphExecDestroy(w.cyc); w.cyc = nullptr; }
  w.cyc_key.clear();
  sync();
}

// --------------------------------------------------------------------------
// field operations
// --------------------------------------------------------------------------
template <typename T, bool CJ>
static void launch_march_cj(int grid, cudaStream_t st, const LevelView<T> &L, int mode, T wj,
                            const typename cplx<T>::t *x, const typename cplx<T>::t *b, typename cplx<T>::t *y) {
  switch (mode) {
    case FM_APPLY: k_field_op_march<T, CJ, FM_APPLY><<<grid, MARCH_THREADS, 0, st>>>(L, wj, x, b, y); break;
    case FM_RESID: k_field_op_march<T, CJ, FM_RESID><<<grid, MARCH_THREADS, 0, st>>>(L, wj, x, b, y); break;
    case FM_JACOBI: k_field_op_march<T, CJ, FM_JACOBI><<<grid, MARCH_THREADS, 0, st>>>(L, wj, x, b, y); break;
    default: k_field_op_march<T, CJ, FM_JACOBI0><<<grid, MARCH_THREADS, 0, st>>>(L, wj, x, b, y); break;
  }
}

template <typename T>
void Ctx::field_op(int mode, int cj, T wj, const typename cplx<T>::t *x, const typename cplx<T>::t *b,
                   typename cplx<T>::t *y, bool opA, int level) {
  LevelView<T> L = opA ? viewA<T>() : viewM<T>(level);
  // column strips exist on level 0 and on every other global level (< ls),
  // the only levels this is called on
  if (L.n_strips == 0) fail(FWI_E_INVAL, "internal: no column strips on a global multigrid level");
  const int grid = (L.n_strips + MARCH_THREADS / 32 - 1) / (MARCH_THREADS / 32);
  KPROF(mode == FM_APPLY ? "k_field_op_march:apply" : mode == FM_RESID ? "k_field_op_march:resid" : mode == FM_JACOBI ? "k_field_op_march:jacobi" : "k_field_op_march:jacobi0", opA ? 0 : level, (mode == FM_APPLY || mode == FM_JACOBI0 ? 2.0 : 3.0) * sizeof(typename cplx<T>::t) * lv[opA ? 0 : level].field, st);
  if (cj) launch_march_cj<T, true>(grid, st, L, mode, wj, x, b, y);
  else launch_march_cj<T, false>(grid, st, L, mode, wj, x, b, y);
  KCHECK();
}

// Live timing of the level-0 complex64 two-sweep smoother launches that are
// not being captured into a graph (CUDA events on the context's stream; the
// kernel counts the nodes it processed into L.work).
template <typename T>
bool Ctx::timer_begin(int level, LevelView<T> &L) {
  if (!timer_on || timer_blocked || level != 0 || sizeof(T) != 4) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  CK(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return false;
  if (!ev_work.p) {
    ev_work.alloc(4096);
    ev_work.zero(st);
  }
  if (ev_used == ev_a.size()) {
    cudaEvent_t a, b2;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b2));
    ev_a.push_back(a); ev_b.push_back(b2); ev_bytes.push_back(0.0); ev_pbytes.push_back(0.0);
  }
  L.work = ev_work.p + ev_used;
  CK(cudaEventRecord(ev_a[ev_used], st));
  return true;
}

void Ctx::timer_end(int streams, int pass_streams, size_t elem_bytes) {
  CK(cudaEventRecord(ev_b[ev_used], st));
  ev_bytes[ev_used] = (double)streams * (double)elem_bytes;
  ev_pbytes[ev_used] = (double)pass_streams * (double)elem_bytes;
  ++ev_used;
  if (ev_used >= 4096) sync();
}

// y = A' x (cj: A'^H) on level 0 with nd = 1: partial_s[strip][0] = <a, y>,
// nd = 2: <y, a>, <y, y> (per-strip shares of the BiCGStab dot products).
template <typename T>
void Ctx::apply_dots(int cj, const typename cplx<T>::t *x, typename cplx<T>::t *y, const typename cplx<T>::t *a,
                     int nd) {
  LevelView<T> L = viewA<T>();
  const int grid = std::max(1, (L.n_strips + MARCH_THREADS / 32 - 1) / (MARCH_THREADS / 32));
  const T w = 0;
  KPROF("k_field_op_march:apply+dots", 0, 3.0 * sizeof(typename cplx<T>::t) * F0, st);
  if (nd == 1) {
    if (cj) k_field_op_march<T, true, FM_APPLY, 1><<<grid, MARCH_THREADS, 0, st>>>(L, w, x, a, y, partial_s.p);
    else k_field_op_march<T, false, FM_APPLY, 1><<<grid, MARCH_THREADS, 0, st>>>(L, w, x, a, y, partial_s.p);
  } else {
    if (cj) k_field_op_march<T, true, FM_APPLY, 2><<<grid, MARCH_THREADS, 0, st>>>(L, w, x, a, y, partial_s.p);
    else k_field_op_march<T, false, FM_APPLY, 2><<<grid, MARCH_THREADS, 0, st>>>(L, w, x, a, y, partial_s.p);
  }
  KCHECK();
}

// Two damped-Jacobi sweeps in one pass on a fine level (x == nullptr: the
// first sweep starts from zero); y must not alias x or b.
template <typename T>
void Ctx::jacobi2(int cj, T wj, const typename cplx<T>::t *x, const typename cplx<T>::t *b,
                  typename cplx<T>::t *y, int level, const BFuse<T> *fz) {
  typedef typename cplx<T>::t T2c;
  LevelView<T> L = viewM<T>(level);
  const bool timed = timer_begin<T>(level, L);
  const int grid = std::max(1, (L.n_strips2 + MARCH_THREADS / 32 - 1) / (MARCH_THREADS / 32));
  // complex64 passes that form the BiCGStab update on the fly (three or four
  // input streams): the input rows staged in shared memory by asynchronous
  // copies (k_jacobi2_stage, 147 -> 99 us per level-0 launch); the other
  // passes and complex128: the register pipeline (k_jacobi2_march), which is
  // faster for them (85 vs 93 us at level 0, 30.5 vs 33.4 us at level 1)
  auto launch = [&](auto zero_t, auto bf_t, const T2c *xx, const T2c *bbv) {
    constexpr bool Z = decltype(zero_t)::value;
    constexpr int F = decltype(bf_t)::value;
    if constexpr (sizeof(T) == 4 && F != 0) {
      constexpr size_t sm = j2_stage_bytes<Z, F>();
      // the dynamic shared-memory limit is raised once per device and variant
      static std::atomic<unsigned long long> attr[2];
      const unsigned long long bit = 1ull << (dev & 63);
      if (!(attr[cj ? 1 : 0].load() & bit)) {
        if (cj) CK(cudaFuncSetAttribute(k_jacobi2_stage<T, true, Z, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        else CK(cudaFuncSetAttribute(k_jacobi2_stage<T, false, Z, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr[cj ? 1 : 0].fetch_or(bit);
      }
      if (cj) k_jacobi2_stage<T, true, Z, F><<<grid, MARCH_THREADS, sm, st>>>(L, wj, xx, bbv, y, fz ? *fz : BFuse<T>{});
      else k_jacobi2_stage<T, false, Z, F><<<grid, MARCH_THREADS, sm, st>>>(L, wj, xx, bbv, y, fz ? *fz : BFuse<T>{});
    } else {
      if (cj) k_jacobi2_march<T, true, Z, F><<<grid, MARCH_THREADS, 0, st>>>(L, wj, xx, bbv, y, fz ? *fz : BFuse<T>{});
      else k_jacobi2_march<T, false, Z, F><<<grid, MARCH_THREADS, 0, st>>>(L, wj, xx, bbv, y, fz ? *fz : BFuse<T>{});
    }
  };
  if (fz) {
    // first pass from zero with the BiCGStab update formed on the fly (b = fz->out)
    const int bf = fz->pold ? 1 : 2;
    KPROF(bf == 1 ? "k_jacobi2_march+p_update" : "k_jacobi2_march+s_update", level,
          (5.0 + (bf == 1 ? 4.0 : 3.0)) * sizeof(typename cplx<T>::t) * lv[level].field, st);
    if (bf == 1) launch(std::true_type{}, std::integral_constant<int, 1>{}, nullptr, nullptr);
    else launch(std::true_type{}, std::integral_constant<int, 2>{}, nullptr, nullptr);
    KCHECK();
    // algorithmic bytes per node: the update's operands (r, v, old p) and result,
    // then the two sweeps (b and the result, x and b and the result); the pass
    // itself reads r, v (and old p) and writes b and y
    if (timed) timer_end(5 + (bf == 1 ? 4 : 3), bf == 1 ? 5 : 4, sizeof(typename cplx<T>::t));
    return;
  }
  KPROF("k_jacobi2_march", level, (x == nullptr ? 5.0 : 6.0) * sizeof(typename cplx<T>::t) * lv[level].field, st);
  if (x == nullptr) launch(std::true_type{}, std::integral_constant<int, 0>{}, x, b);
  else launch(std::false_type{}, std::integral_constant<int, 0>{}, x, b);
  KCHECK();
  // algorithmic bytes per node: x, b and the result of each of the two sweeps
  // (the first sweep from zero reads no x); the fused pass itself reads b
  // (and x) and writes y once
  if (timed) timer_end(x == nullptr ? 5 : 6, x == nullptr ? 2 : 3, sizeof(typename cplx<T>::t));
}

// b_{l+1} = P^T (b_l - M_l x_l) on every block.
template <typename T>
void Ctx::resid_restrict(int cj, int l, const typename cplx<T>::t *x, const typename cplx<T>::t *b,
                         typename cplx<T>::t *bc) {
  LevelView<T> Lf = viewM<T>(l), Lc = viewM<T>(l + 1);
  const int n = lv[l].n_rstrips;   // built for every global level l < ls, the only levels that restrict
  if (n == 0) fail(FWI_E_INVAL, "internal: no restriction strips on a global multigrid level");
  const int grid = (n + MARCH_THREADS / 32 - 1) / (MARCH_THREADS / 32);
  // complex64 level 0 (HBM-resident, latency of the row loads): rows staged in
  // shared memory by asynchronous copies; the L2-resident coarser levels and
  // complex128 keep the register pipeline (faster there)
  const bool staged = sizeof(T) == 4 && l == 0;
  KPROF(staged ? "k_resid_restrict_stage" : "k_resid_restrict_march", l,
        sizeof(typename cplx<T>::t) * (2.0 * lv[l].field + lv[l + 1].field), st);
  if constexpr (sizeof(T) == 4) {
    if (staged) {
      if (cj) k_resid_restrict_stage<T, true><<<grid, MARCH_THREADS, 0, st>>>(Lf, Lc, x, b, bc, lv[l].rstrips.p, n);
      else k_resid_restrict_stage<T, false><<<grid, MARCH_THREADS, 0, st>>>(Lf, Lc, x, b, bc, lv[l].rstrips.p, n);
    }
  }
  if (!staged) {
    if (cj) k_resid_restrict_march<T, true><<<grid, MARCH_THREADS, 0, st>>>(Lf, Lc, x, b, bc, lv[l].rstrips.p, n);
    else k_resid_restrict_march<T, false><<<grid, MARCH_THREADS, 0, st>>>(Lf, Lc, x, b, bc, lv[l].rstrips.p, n);
  }
  KCHECK();
}

// x_l += P x_{l+1} (bilinear) on every block.
template <typename T>
void Ctx::prolong(int l, const LevelView<T> &Lf, const LevelView<T> &Lc, const typename cplx<T>::t *xc,
                  typename cplx<T>::t *xf) {
  const int n = lv[l].n_pstrips;   // built with the restriction strips
  if (n == 0) fail(FWI_E_INVAL, "internal: no prolongation strips on a global multigrid level");
  const int grid = (n + MARCH_THREADS / 32 - 1) / (MARCH_THREADS / 32);
  KPROF("k_prolong_march", l, sizeof(typename cplx<T>::t) * (2.0 * lv[l].field + lv[l + 1].field), st);
  k_prolong_march<T><<<grid, MARCH_THREADS, 0, st>>>(Lf, Lc, xc, xf, lv[l].pstrips.p, n);
  KCHECK();
}

template <typename T>
void Ctx::block_dots(int nd, const typename cplx<T>::t *a0, const typename cplx<T>::t *b0,
                     const typename cplx<T>::t *a1, const typename cplx<T>::t *b1,
                     const typename cplx<T>::t *a2, const typename cplx<T>::t *b2) {
  LevelView<T> L = viewA<T>();
  KPROF("k_block_dots", 0, 2.0 * nd * sizeof(typename cplx<T>::t) * F0, st);
  k_block_dots<T><<<L.n_tiles, TILE_THREADS, 0, st>>>(L, nd, a0, b0, a1, b1, a2, b2, partial.p);
  KCHECK();
}

// One multigrid cycle for the shifted operator, x = cycle(b) (Sec. 5: the
// shifted-Laplacian preconditioner; levels >= ls run in shared memory).
// nu damped-Jacobi sweeps on level l (from x = 0 when zero, else from cur);
// the result ends in cur (oth is the other buffer).  Sweeps go in fused pairs
// on the fine levels.
template <typename T>
void Ctx::smooth(int nu, bool zero, int cj, T wj, const typename cplx<T>::t *bl, typename cplx<T>::t *&cur,
                 typename cplx<T>::t *&oth, int l, const BFuse<T> *fz) {
  int s = 0;
  if (lv[l].n_strips2 > 0) {
    if (zero && nu >= 2) {
      jacobi2<T>(cj, wj, nullptr, bl, cur, l, fz);
      s = 2;
    }
    for (; s + 1 < nu; s += 2) {
      jacobi2<T>(cj, wj, cur, bl, oth, l);
      std::swap(cur, oth);
    }
  }
  for (; s < nu; ++s) {
    if (zero && s == 0) {
      field_op<T>(FM_JACOBI0, cj, wj, nullptr, bl, cur, false, l);
    } else {
      field_op<T>(FM_JACOBI, cj, wj, cur, bl, oth, false, l);
      std::swap(cur, oth);
    }
  }
}

template <typename T>
void Ctx::mg_cycle(const typename cplx<T>::t *b, typename cplx<T>::t *x, int cj, const fwi_opts &o,
                   const BFuse<T> *fz) {
  typedef typename cplx<T>::t T2;
  Work<T> &w = work<T>();
  // a BiCGStab update fused into the first level-0 pass needs that pass to be
  // a two-sweep pass from zero on the global level 0; otherwise form it first
  if (fz && !(ls_p[sizeof(T) == 8] > 0 && o.nu1 >= 2 && lv[0].n_strips2 > 0)) {
    bicg_update_into<T>(*fz);
    fz = nullptr;
  }
  const T wj = (T)o.omega_jac;
  CoarseArgs ca;
  for (int l = 0; l < MAX_LEVELS; ++l) ca.blks[l] = l < nlev_max ? lv[l].blksM.p : nullptr;
  ca.ops = d_ops.p; ca.inv = inv.p; ca.inv_off = inv_off.p; ca.inst_nlev = d_inst_nlev.p;
  ca.skip = cur_skip;
  const int ls = ls_p[sizeof(T) == 8];
  ca.ls = ls; ca.nu1 = o.nu1; ca.nu2 = o.nu2; ca.cyc = o.mg_cycle; ca.cj = cj; ca.w = o.omega_jac;
  ca.wdepth = o.mg_wdepth;
  size_t smem = smem_bytes[sizeof(T) == 8];
  if (ls == 0) {
    launch_coarse<T>(ca, smem, b, x, cj, o.coarse_threads);
    return;
  }
  // recursive cycle over the global levels 0..ls-1; returns the buffer that
  // holds the level's solution.
  std::function<T2 *(int, const T2 *, T2 *, T2 *)> cyc;
  cyc = [&](int l, const T2 *bl, T2 *xa, T2 *xb) -> T2 * {
    if (l == ls) {
      launch_coarse<T>(ca, smem, bl, xa, cj, o.coarse_threads);
      return xa;
    }
    T2 *cur = xa, *oth = xb;
    if (o.nu1 == 0) CK(cudaMemsetAsync(cur, 0, lv[l].field * sizeof(T2), st));
    smooth<T>(o.nu1, true, cj, wj, bl, cur, oth, l, l == 0 ? fz : nullptr);
    int reps = (l > 0 && l <= o.mg_wdepth) ? o.mg_cycle : 1;
    for (int r = 0; r < reps; ++r) {
      LevelView<T> Lf = viewM<T>(l), Lc = viewM<T>(l + 1);
      resid_restrict<T>(cj, l, cur, bl, w.lb[l + 1].p);
      T2 *xc = cyc(l + 1, w.lb[l + 1].p, w.lx[l + 1].p, w.lt[l + 1].p);
      prolong<T>(l, Lf, Lc, xc, cur);
    }
    smooth<T>(o.nu2, false, cj, wj, bl, cur, oth, l);
    return cur;
  };
  T2 *res = cyc(0, b, x, w.t0a.p);
  if (res != x) CK(cudaMemcpyAsync(x, res, F0 * sizeof(T2), cudaMemcpyDeviceToDevice, st));
}

// The same cycle as mg_cycle, with every level buffer supplied by the caller
// (used by fwi_mg_cycle_noalloc, whose buffers live in a static device array).
template <typename T>
void Ctx::mg_cycle_into(const typename cplx<T>::t *b, typename cplx<T>::t *x, int cj, const fwi_opts &o,
                        typename cplx<T>::t *const *lx, typename cplx<T>::t *const *lb,
                        typename cplx<T>::t *const *lt, typename cplx<T>::t *t0) {
  typedef typename cplx<T>::t T2;
  const T wj = (T)o.omega_jac;
  CoarseArgs ca;
  for (int l = 0; l < MAX_LEVELS; ++l) ca.blks[l] = l < nlev_max ? lv[l].blksM.p : nullptr;
  ca.ops = d_ops.p; ca.inv = inv.p; ca.inv_off = inv_off.p; ca.inst_nlev = d_inst_nlev.p;
  ca.skip = cur_skip;
  const int ls = ls_p[sizeof(T) == 8];
  ca.ls = ls; ca.nu1 = o.nu1; ca.nu2 = o.nu2; ca.cyc = o.mg_cycle; ca.cj = cj; ca.w = o.omega_jac;
  ca.wdepth = o.mg_wdepth;
  size_t smem = smem_bytes[sizeof(T) == 8];
  if (ls == 0) {
    launch_coarse<T>(ca, smem, b, x, cj, o.coarse_threads);
    return;
  }
  std::function<T2 *(int, const T2 *, T2 *, T2 *)> cyc;
  cyc = [&](int l, const T2 *bl, T2 *xa, T2 *xb) -> T2 * {
    if (l == ls) {
      launch_coarse<T>(ca, smem, bl, xa, cj, o.coarse_threads);
      return xa;
    }
    T2 *cur = xa, *oth = xb;
    if (o.nu1 == 0) CK(cudaMemsetAsync(cur, 0, lv[l].field * sizeof(T2), st));
    smooth<T>(o.nu1, true, cj, wj, bl, cur, oth, l);
    int reps = (l > 0 && l <= o.mg_wdepth) ? o.mg_cycle : 1;
    for (int r = 0; r < reps; ++r) {
      LevelView<T> Lf = viewM<T>(l), Lc = viewM<T>(l + 1);
      resid_restrict<T>(cj, l, cur, bl, lb[l + 1]);
      T2 *xc = cyc(l + 1, lb[l + 1], lx[l + 1], lt[l + 1]);
      prolong<T>(l, Lf, Lc, xc, cur);
    }
    smooth<T>(o.nu2, false, cj, wj, bl, cur, oth, l);
    return cur;
  };
  T2 *res = cyc(0, b, x, t0);
  if (res != x) CK(cudaMemcpyAsync(x, res, F0 * sizeof(T2), cudaMemcpyDeviceToDevice, st));
}

// The BiCGStab update of a fused descriptor as separate passes (for cycles
// whose first level-0 pass cannot form it): out = r + beta (pold - omega v)
// or out = r - alpha v.
template <typename T>
void Ctx::bicg_update_into(const BFuse<T> &fz) {
  typedef typename cplx<T>::t T2;
  LevelView<T> L = viewA<T>();
  const int nt = L.n_tiles;
  if (fz.pold) {
    if (fz.pold != fz.out) {
      KPROF("k_bicg_update", 3, 2.0 * sizeof(T2) * F0, st);
      k_bicg_update<T, 3><<<nt, TILE_THREADS, 0, st>>>(L, fz.S, fz.out, fz.pold, nullptr);
      KCHECK();
    }
    KPROF("k_bicg_update", 0, 4.0 * sizeof(T2) * F0, st);
    k_bicg_update<T, 0><<<nt, TILE_THREADS, 0, st>>>(L, fz.S, fz.out, fz.r, fz.v);
    KCHECK();
  } else {
    KPROF("k_bicg_update", 1, 3.0 * sizeof(T2) * F0, st);
    k_bicg_update<T, 1><<<nt, TILE_THREADS, 0, st>>>(L, fz.S, fz.out, fz.r, fz.v);
    KCHECK();
  }
}

// ILU(0) factors of every A operator (level 0, one per instance and
// frequency), built once per hierarchy (models and options).
void Ctx::ensure_ilu() {
  if (ilu_key == hier_key && ilu64.p) return;
  std::vector<int> ids;
  std::vector<long long> offs(h_ops.size(), -1), foff;
  long long tot = 0;
  int maxnz = 1;
  for (int b = 0; b < B; ++b) {
    const int id = lv[0].hA[b].op;
    if (offs[id] >= 0) continue;
    offs[id] = tot;
    ids.push_back(id);
    foff.push_back(tot);
    tot += (long long)h_ops[id].nx * h_ops[id].nz;
    maxnz = std::max(maxnz, h_ops[id].nz);
  }
  ilu64.alloc(5 * tot);
  ilu32.alloc(5 * tot);
  ilu_off.upload(offs, st);
  ilu_stride = tot;
  ilu_maxnz = maxnz;
  DBuf<int> dids;
  DBuf<long long> dfo;
  dids.upload(ids, st);
  dfo.upload(foff, st);
  const int nth = std::min(1024, (maxnz + 31) / 32 * 32);
  const size_t smem = 2 * (size_t)maxnz * sizeof(double2);
  KPROF("k_ilu_factor", -1, 0, st);
  k_ilu_factor<<<(int)ids.size(), nth, smem, st>>>(d_ops.p, dids.p, dfo.p, st64.p, gam64.p, ilu64.p, ilu32.p, tot);
  KCHECK();
  sync();
  ilu_key = hier_key;
}

template <typename T> static const typename cplx<T>::t *ilu_ptr(Ctx &c);
template <> const float2 *ilu_ptr<float>(Ctx &c) { return c.ilu32.p; }
template <> const double2 *ilu_ptr<double>(Ctx &c) { return c.ilu64.p; }

// x = (L U)^{-1} b (cj: the adjoint approximation) for every block.
template <typename T>
void Ctx::ilu_apply(int cj, const typename cplx<T>::t *b, typename cplx<T>::t *x) {
  typedef typename cplx<T>::t T2;
  // the factors are built before any stream capture (ensure_ilu allocates,
  // uploads and synchronises); here they must already exist
  if (!(ilu_key == hier_key && ilu64.p)) fail(FWI_E_INVAL, "internal: ILU(0) factors not built before use");
  const int nth = std::min(1024, (ilu_maxnz + 31) / 32 * 32);
  const size_t smem = 2 * (size_t)ilu_maxnz * sizeof(T2);
  KPROF("k_ilu_solve", 0, 4.0 * sizeof(T2) * F0, st);
  if (cj) k_ilu_solve<T, true><<<B, nth, smem, st>>>(lv[0].blksA.p, d_ops.p, ilu_off.p, ilu_ptr<T>(*this), ilu_stride,
                                                    cur_skip, b, x);
  else k_ilu_solve<T, false><<<B, nth, smem, st>>>(lv[0].blksA.p, d_ops.p, ilu_off.p, ilu_ptr<T>(*this), ilu_stride,
                                                  cur_skip, b, x);
  KCHECK();
}

// Batched right-preconditioned BiCGStab, one independent system per block
// (per-block scalars), x = approx A'^{-1} b (cj = 1: A'^H).
template <typename T>
void Ctx::inner_solve(const typename cplx<T>::t *b, typename cplx<T>::t *x, int cj, int iters, double tol,
                      const fwi_opts &o, long long *count, bool ilu) {
  typedef typename cplx<T>::t T2;
  Work<T> &w = work<T>();
  LevelView<T> L = viewA<T>();
  const int nt = L.n_tiles;
  const int sb = (B + BICG_WARPS - 1) / BICG_WARPS;
  auto upd = [&](int opk, T2 *y, const T2 *a, const T2 *c) {
    KPROF("k_bicg_update", opk, (opk == 0 ? 4.0 : opk == 1 ? 3.0 : opk == 3 ? 2.0 : 1.0) * sizeof(T2) * F0, st);
    // complex64 with 16-byte aligned vectors: two nodes per access over each row tile
    constexpr bool V4 = sizeof(T) == 4;
    const bool vec = V4 && aligned16({y, a, c});
    if (opk == 0) {
      if (vec) k_bicg_update<T, 0, V4><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
      else k_bicg_update<T, 0><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
    } else if (opk == 1) {
      if (vec) k_bicg_update<T, 1, V4><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
      else k_bicg_update<T, 1><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
    } else if (opk == 3) {
      if (vec) k_bicg_update<T, 3, V4><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
      else k_bicg_update<T, 3><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
    } else {
      if (vec) k_bicg_update<T, 4, V4><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
      else k_bicg_update<T, 4><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, y, a, c);
    }
    KCHECK();
  };
  auto scal = [&](int stage) {
    KPROF("k_bicg_scalars", -1, 0, st);
    k_bicg_scalars<<<sb, BICG_WARPS * 32, 0, st>>>(B, lv[0].t0.p, lv[0].t1.p, partial.p, w.bst.p, stage, tol, w.done.p);
    KCHECK();
  };
  // stages whose dots come from the strip kernels (operator apply fused with dots)
  auto scal_s = [&](int stage) {
    KPROF("k_bicg_scalars", -1, 0, st);
    k_bicg_scalars<<<sb, BICG_WARPS * 32, 0, st>>>(B, lv[0].s0.p, lv[0].s1.p, partial_s.p, w.bst.p, stage, tol, w.done.p);
    KCHECK();
  };
  // x = 0, r = b, rh = b, p = v = 0
  upd(4, x, nullptr, nullptr);
  upd(3, w.r.p, b, nullptr);
  upd(3, w.rh.p, b, nullptr);
  upd(4, w.p.p, nullptr, nullptr);
  upd(4, w.v.p, nullptr, nullptr);
  block_dots<T>(1, b, b, nullptr, nullptr, nullptr, nullptr);
  scal(0);
  // from here on, kernels skip the blocks whose solve has finished (zero
  // right-hand side, breakdown, or tolerance reached): their x and r no longer
  // change, exactly as when the iteration stops
  struct SkipGuard {
    Ctx &c;
    ~SkipGuard() { c.cur_skip = nullptr; }
  } guard{*this};
  cur_skip = w.done.p;
  L = viewA<T>();
  // rho = <rh, r> = <b, b> for the first iteration: the partials still hold <b, b>
  scal(1);
  // the p update is formed inside the first smoothing pass of the cycle that
  // consumes it (its separate pass was the slower one; the s update stays a
  // separate pass, which costs less than the loads it would add to the
  // latency-bound smoother); p alternates between two buffers because that
  // pass reads the previous p around its strips while writing the new one
  T2 *pc = w.p.p, *pn = w.p2.p;
  for (int it = 0; it < iters; ++it) {
    const BFuse<T> fp{w.r.p, w.v.p, pc, pn, w.bst.p};                 // p = r + beta (p - omega v)
    if (ilu) {                                                         // ph = K p
      bicg_update_into<T>(fp);
      ilu_apply<T>(cj, pn, w.ph.p);
    } else {
      mg_cycle<T>(pn, w.ph.p, cj, o, &fp);
    }
    std::swap(pc, pn);
    apply_dots<T>(cj, w.ph.p, w.v.p, w.rh.p, 1);                       // v = A ph, <rh, v>
    scal_s(2);
    upd(1, w.s.p, w.r.p, w.v.p);                                       // s = r - alpha v
    if (ilu) ilu_apply<T>(cj, w.s.p, w.sh.p);                          // sh = K s
    else mg_cycle<T>(w.s.p, w.sh.p, cj, o);
    apply_dots<T>(cj, w.sh.p, w.t.p, w.s.p, 2);                        // t = A sh, <t, s>, <t, t>
    scal_s(3);
    // x += alpha ph + omega sh; r = s - omega t; <r, r>, <rh, r>
    KPROF("k_bicg_xr", 0, 8.0 * sizeof(typename cplx<T>::t) * F0, st);
    if (sizeof(T) == 4 && aligned16({x, w.ph.p, w.sh.p, w.s.p, w.r.p, w.t.p, w.rh.p}))
      k_bicg_xr<T, sizeof(T) == 4><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, x, w.ph.p, w.sh.p, w.s.p, w.r.p, w.t.p,
                                                                w.rh.p, partial.p);
    else
      k_bicg_xr<T, false><<<nt, TILE_THREADS, 0, st>>>(L, w.bst.p, x, w.ph.p, w.sh.p, w.s.p, w.r.p, w.t.p, w.rh.p,
                                                       partial.p);
    KCHECK();
    scal(5);                                                           // stage 4, then the next stage 1
    if (count) *count += B;
  }
}

// --------------------------------------------------------------------------
// KKT operator (Sec. 4, eq. KKT, rescaled) and preconditioner (Sec. 5)
// --------------------------------------------------------------------------
template <typename T>
void Ctx::kkt_matvec(const T *xi, T *y, double eps, const typename cplx<T>::t *u) {
  typedef typename cplx<T>::t T2;
  const T2 *du = (const T2 *)xi;
  const T2 *lm = (const T2 *)(xi + 2 * F0);
  const T *ds = xi + 4 * F0;
  T2 *yu = (T2 *)y;
  T2 *ylm = (T2 *)(y + 2 * F0);
  T *ys = y + 4 * F0;
  LevelView<T> L = viewA<T>();
  KPROF("k_kkt_rows", 0, 5.0 * sizeof(typename cplx<T>::t) * F0, st);
  k_kkt_rows<T><<<L.n_tiles, TILE_THREADS, 0, st>>>(L, d_inst.p, cfK.p, u, du, lm, ds, yu, ylm);
  KCHECK();
  if (n_F) {
    KPROF("k_kkt_F", 0, 3.0 * sizeof(typename cplx<T>::t) * n_F, st);
    k_kkt_F<T><<<grid_for(n_F, 128, 1 << 20), 128, 0, st>>>(n_F, d_F_node.p, d_F_w2.p, du, yu);
    KCHECK();
  }
  long long mx = 0;
  for (auto &I : inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
  dim3 g((unsigned)((mx + 127) / 128), (unsigned)inst.size());
  KPROF("k_coupling_reduce", 0, 2.0 * sizeof(typename cplx<T>::t) * cpl_nodes() + 2.0 * sizeof(T) * Nc, st);
  k_coupling_reduce<T, T><<<g, dim3(128, CPL_ROWS), 0, st>>>(d_inst.p, d_blk_off.p, cfK.p, u, lm, ds, eps, 0, ys);
  KCHECK();
}

static_assert(QN_MAX == FWI_HBLOCK_MAX, "pair capacity of the H-block kernels");

// Quasi-Newton H block (Sec. 5 after eq. precond; Sec. 7): m pairs (s_j, y_j)
// of the scaled control, oldest first, with s_j^T y_j > 0.  The pairs are
// copied; their Gram matrices S^T Y and Y^T Y are formed once here (FP64).
void Ctx::hblock_set(int m, const double *S, const double *Y, int on_device) {
  if (m < 0 || m > QN_MAX) fail(FWI_E_INVAL, "hblock: m must be in 0 .. FWI_HBLOCK_MAX");
  if (!layout_ok || Nc <= 0) fail(FWI_E_INVAL, "hblock: set the surveys first (the control size is not known)");
  ++qn_version;
  qn_eps = 0.0;
  if (m == 0) { qn_m = 0; return; }
  if (!S || !Y) fail(FWI_E_INVAL, "hblock: null pair buffer");
  const size_t n = (size_t)m * Nc;
  qnS.alloc(n); qnY.alloc(n);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(qnS.p, S, n * sizeof(double), kind, st));
  CK(cudaMemcpyAsync(qnY.p, Y, n * sizeof(double), kind, st));
  const int g = qn_grid();
  qnPart.alloc((size_t)FLAT_BLOCKS * 2 * QN_MAX);
  qn_SY.assign((size_t)m * m, 0.0);
  qn_YY.assign((size_t)m * m, 0.0);
  std::vector<double> hp((size_t)g * 2 * QN_MAX);
  for (int k = 0; k < m; ++k) {
    // column k: s_j^T y_k and y_j^T y_k for every j
    KPROF("k_qn_dots", -1, 8.0 * (2 * m + 1) * Nc, st);
    k_qn_dots<double><<<g, FLAT_THREADS, 0, st>>>(Nc, qnY.p + (size_t)k * Nc, qnS.p, qnY.p, m, qnPart.p);
    KCHECK();
    CK(cudaMemcpyAsync(hp.data(), qnPart.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    for (int j = 0; j < m; ++j) {
      double a = 0.0, b = 0.0;
      for (int p = 0; p < g; ++p) { a += hp[(size_t)p * 2 * QN_MAX + j]; b += hp[(size_t)p * 2 * QN_MAX + QN_MAX + j]; }
      qn_SY[(size_t)j * m + k] = a;
      qn_YY[(size_t)j * m + k] = b;
    }
  }
  for (int j = 0; j < m; ++j) {
    const double c = qn_SY[(size_t)j * m + j];
    if (!(c > 0.0) || !std::isfinite(c)) {
      qn_m = 0;
      fail(FWI_E_INVAL, "hblock: pair " + std::to_string(j) + " has no positive curvature (s^T y <= 0)");
    }
  }
  qn_m = m;
}

// Fold the compact form for this eps: with q = t / eps (what the
// preconditioner has formed), B^{-1} t = q + S c_S + Y c_Y, c = Mf [S^T q; Y^T q],
//   Mf = [[eps R^-T (D + Y^T Y / eps) R^-1, -R^-T], [-R^-1, 0]].
void Ctx::hblock_prepare(const fwi_opts &o) {
  if (!o.hblock || qn_m == 0 || qn_eps == o.eps) return;
  const int m = qn_m;
  const double eps = o.eps, gam = 1.0 / o.eps;
  // Ri = R^{-1}, R the upper triangle of S^T Y (back substitution, column by column)
  std::vector<double> Ri((size_t)m * m, 0.0);
  auto R = [&](int i, int j) { return qn_SY[(size_t)i * m + j]; };
  for (int c = 0; c < m; ++c)
    for (int i = c; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = i + 1; k <= c; ++k) v -= R(i, k) * Ri[(size_t)k * m + c];
      Ri[(size_t)i * m + c] = v / R(i, i);
    }
  // C1 = Ri^T (D + gam YY) Ri
  std::vector<double> Mid((size_t)m * m), T1((size_t)m * m, 0.0), C1((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Mid[(size_t)i * m + j] = gam * qn_YY[(size_t)i * m + j] + (i == j ? R(i, i) : 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double v = 0.0;
      for (int k = 0; k < m; ++k) v += Mid[(size_t)i * m + k] * Ri[(size_t)k * m + j];
      T1[(size_t)i * m + j] = v;
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double v = 0.0;
      for (int k = 0; k < m; ++k) v += Ri[(size_t)k * m + i] * T1[(size_t)k * m + j];
      C1[(size_t)i * m + j] = v;
    }
  std::vector<double> Mf((size_t)4 * m * m, 0.0);
  const int w = 2 * m;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      Mf[(size_t)i * w + j] = eps * C1[(size_t)i * m + j];
      Mf[(size_t)i * w + m + j] = -Ri[(size_t)j * m + i];       // -R^{-T}
      Mf[(size_t)(m + i) * w + j] = -Ri[(size_t)i * m + j];     // -R^{-1}
    }
  qnMf.upload(Mf, st);
  sync();
  qn_eps = o.eps;
}

template <typename T> void Ctx::hblock_apply(T *zs, const fwi_opts &o) {
  if (!o.hblock || qn_m == 0) return;
  if (qn_eps != o.eps) fail(FWI_E_CUDA, "internal: H block not prepared for this eps");
  const int g = qn_grid();
  KPROF("k_qn_dots", 0, (double)sizeof(T) * Nc + 16.0 * qn_m * Nc, st);
  k_qn_dots<T><<<g, FLAT_THREADS, 0, st>>>(Nc, zs, qnS.p, qnY.p, qn_m, qnPart.p);
  KCHECK();
  KPROF("k_qn_apply", 0, 2.0 * sizeof(T) * Nc + 16.0 * qn_m * Nc, st);
  k_qn_apply<T><<<g, FLAT_THREADS, 0, st>>>(Nc, zs, qnS.p, qnY.p, qn_m, qnPart.p, g, qnMf.p);
  KCHECK();
}

template <typename T>
void Ctx::precond(const T *v, T *z, const fwi_opts &o, long long *count, const typename cplx<T>::t *u) {
  typedef typename cplx<T>::t T2;
  Work<T> &w = work<T>();
  const T2 *v1 = (const T2 *)v;
  const T2 *v3 = (const T2 *)(v + 2 * F0);
  const T *v2 = v + 4 * F0;
  T2 *zu = (T2 *)z;
  T2 *zl = (T2 *)(z + 2 * F0);
  T *zs = z + 4 * F0;
  int iters = o.inner_iters;
  double tol = o.inner_tol;
  if (tol > 0.0) iters = std::max(iters, 2000);
  // z_lambda = A'^{-H} v1 (inner_solver 2: one ILU(0) application, the paper's A~)
  if (o.inner_solver == 2) ilu_apply<T>(1, v1, zl);
  else inner_solve<T>(v1, zl, 1, iters, tol, o, count, o.inner_solver == 1);
  // z_s = (v2 + Re(P~^H z_lambda)) / eps
  long long mx = 0;
  for (auto &I : inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
  dim3 g((unsigned)((mx + 127) / 128), (unsigned)inst.size());
  KPROF("k_coupling_reduce", 1, 2.0 * sizeof(typename cplx<T>::t) * cpl_nodes() + 2.0 * sizeof(T) * Nc, st);
  k_coupling_reduce<T, T><<<g, dim3(128, CPL_ROWS), 0, st>>>(d_inst.p, d_blk_off.p, cfK.p, u, zl, v2, o.eps, 1, zs);
  KCHECK();
  // quasi-Newton H block: z_s = B^{-1} (v2 + Re(P~^H z_lambda)) instead of ( ) / eps
  hblock_apply<T>(zs, o);
  // z_u = A'^{-1} (v3 + P~ z_s)
  LevelView<T> L = viewA<T>();
  KPROF("k_coupling_scatter", 0, 3.0 * sizeof(typename cplx<T>::t) * F0, st);
  k_coupling_scatter<T><<<L.n_tiles, TILE_THREADS, 0, st>>>(L, d_inst.p, cfK.p, u, v3, zs, w.t0b.p);
  KCHECK();
  if (o.inner_solver == 2) ilu_apply<T>(0, w.t0b.p, zu);
  else inner_solve<T>(w.t0b.p, zu, 0, iters, tol, o, count, o.inner_solver == 1);
}

// Preconditioner application, replayed from a CUDA graph when requested (the
// graph reads w.vin and writes w.zout).
template <typename T>
void Ctx::precond_any(const T *v, T *z, const fwi_opts &o, long long *count, const typename cplx<T>::t *u) {
  Work<T> &w = work<T>();
  bool graphable = o.use_graph && !(o.inner_tol > 0.0);
  if (!graphable) { precond<T>(v, z, o, count, u); return; }
  char key[256];
  snprintf(key, sizeof key, "%s|%d|%d|%d|%d|%d|%.17g|%.17g|%.17g|%p|%d|%d", hier_key.c_str(), o.inner_iters, o.mg_cycle,
           o.mg_wdepth, o.nu1, o.nu2, o.omega_jac, o.eps, o.shift_beta, (const void *)u, o.coarse_threads * 10 + o.inner_solver,
           hb_key(o));
  if (w.graph_key != key) {
    if (w.graph) { cudaGraphExecDestroy(w.graph); w.graph = nullptr; }
    cudaGraph_t gr;
    unsigned long long before = g_launches.load();
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    long long dummy = 0;
    try {
      precond<T>(w.vin.p, w.zout.p, o, &dummy, u);
    } catch (...) {
      cudaStreamEndCapture(st, &gr);
      throw;
    }
    CK(cudaStreamEndCapture(st, &gr));
    CK(cudaGraphInstantiate(&w.graph, gr, 0));
    cudaGraphDestroy(gr);
    w.graph_key = key;
    w.graph_kernels = g_launches.load() - before;
    g_launches.fetch_sub(w.graph_kernels);   // captured, not launched
  }
  CK(cudaMemcpyAsync(w.vin.p, v, nkkt * sizeof(T), cudaMemcpyDeviceToDevice, st));
  CK(cudaGraphLaunch(w.graph, st));
  g_launches.fetch_add(w.graph_kernels);
  CK(cudaMemcpyAsync(z, w.zout.p, nkkt * sizeof(T), cudaMemcpyDeviceToDevice, st));
  if (count && o.inner_solver != 2) *count += 2LL * o.inner_iters * B;
}

template <typename T>
void Ctx::multidot(long long n, int nv, T *const *dV, const T *wv, double *out, int acc, int pm) {
  Work<T> &w = work<T>();
  for (int c0 = 0; c0 < nv; c0 += MD_CHUNK) {
    int c = std::min(MD_CHUNK, nv - c0);
    KPROF(pm == DOT_FP64 ? "k_multidot:fp64" : pm == DOT_COMP ? "k_multidot:comp" : "k_multidot:runs", -1,
          (double)(c + 1) * n * sizeof(T), st);
    if (pm == DOT_FP64) k_multidot<T, DOT_FP64><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dV + c0, wv, w.partial_flat.p);
    else if (pm == DOT_COMP) k_multidot<T, DOT_COMP><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dV + c0, wv, w.partial_flat.p);
    else k_multidot<T, DOT_RUNS><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dV + c0, wv, w.partial_flat.p);
    KCHECK();
    KPROF("k_reduce_partials", -1, 0, st);
    k_reduce_partials<<<c, 32, 0, st>>>(c, FLAT_BLOCKS, w.partial_flat.p, out + c0, acc);
    KCHECK();
  }
}

// w += sign * sum_v coef[v] V_v over nv vectors, MD_CHUNK per launch.
template <typename T>
void Ctx::multi_axpy(long long n, int nv, T *const *dV, const double *coef, double sign, T *w) {
  for (int c0 = 0; c0 < nv; c0 += MD_CHUNK) {
    const int c = std::min(MD_CHUNK, nv - c0);
    KPROF("k_multi_axpy", -1, (double)(c + 2) * n * sizeof(T), st);
    k_multi_axpy<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dV + c0, coef + c0, sign, w);
    KCHECK();
  }
}

// ||x||^2 or x.y over a flat array into *out (FP64, deterministic).
template <typename T>
static void flat_dot(cudaStream_t st, long long n, const T *x, const T *y, double *partial, double *out,
                     int pm = DOT_RUNS) {
  KPROF(pm == DOT_FP64 ? "k_dot2:fp64" : pm == DOT_COMP ? "k_dot2:comp" : "k_dot2:runs", -1, 2.0 * n * sizeof(T), st);
  if (pm == DOT_FP64) k_dot2<T, DOT_FP64><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, x, y, partial);
  else if (pm == DOT_COMP) k_dot2<T, DOT_COMP><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, x, y, partial);
  else k_dot2<T, DOT_RUNS><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, x, y, partial);
  KCHECK();
  KPROF("k_reduce_partials", -1, 0, st);
  k_reduce_partials<<<1, 32, 0, st>>>(1, FLAT_BLOCKS, partial, out, 0);
  KCHECK();
}

// One restart cycle of FGMRES as a CUDA graph under device control: a WHILE
// node whose body is one Arnoldi step (V[j] to the preconditioner's input,
// the preconditioner, Z[j], the KKT product, classical Gram-Schmidt twice,
// the norm, the Givens update, V[j+1], and k_fgmres_ctl, which advances j and
// sets the node's condition), followed by the back substitution and
// x += Z y.  The step index and the convergence test live in the device
// control block w.ctl; the host reads it once per cycle.  The graph is
// captured once per (hierarchy, options, wavefields) and replayed.
template <typename T>
void Ctx::fgmres_cycle_graph(const fwi_opts &o, double eps, T *x, const typename cplx<T>::t *u) {
  Work<T> &w = work<T>();
  char key[320];
  snprintf(key, sizeof key, "%s|%d|%d|%d|%d|%d|%.17g|%.17g|%.17g|%p|%d|%d|%p|%d|%d", hier_key.c_str(), o.inner_iters,
           o.mg_cycle, o.mg_wdepth, o.nu1, o.nu2, o.omega_jac, eps, o.shift_beta, (const void *)u, w.m,
           o.arnoldi_dots, (void *)x, o.coarse_threads * 10 + o.inner_solver, hb_key(o));
  if (w.cyc && w.cyc_key == key) return;
  if (w.cyc) { cudaGraphExecDestroy(w.cyc); w.cyc = nullptr; }
  const long long n = nkkt;
  const int m = w.m;
  const int pm = o.arnoldi_dots;
  T *const *dV = w.dptrV.p;
  T *const *dZ = w.dptrZ.p;
  FgCtl *c = w.ctl.p;
  const int nchunk = (m + 1 + MD_CHUNK - 1) / MD_CHUNK;
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  struct GraphGuard {
    cudaGraph_t g;
    ~GraphGuard() { cudaGraphDestroy(g); }
  } gguard{g};
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CK(cudaGraphAddNode(&wnode, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  auto dots = [&](double *out) {          // out[0..j] = V[0..j] . wst, chunk by chunk
    for (int q = 0; q < nchunk; ++q) {
      if (pm == DOT_FP64)
        k_multidot_dev<T, DOT_FP64><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, 0, q * MD_CHUNK, dV, w.wst.p,
                                                                          w.partial_flat.p);
      else if (pm == DOT_COMP)
        k_multidot_dev<T, DOT_COMP><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, 0, q * MD_CHUNK, dV, w.wst.p,
                                                                          w.partial_flat.p);
      else
        k_multidot_dev<T, DOT_RUNS><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, 0, q * MD_CHUNK, dV, w.wst.p,
                                                                          w.partial_flat.p);
      KCHECK();
      k_reduce_partials_dev<<<MD_CHUNK, 32, 0, st>>>(c, 0, q * MD_CHUNK, FLAT_BLOCKS, w.partial_flat.p, out);
      KCHECK();
    }
  };
  auto axpys = [&](T *const *VV, int which, const double *coef, double sign, T *y) {
    for (int q = 0; q < nchunk; ++q) {
      k_multi_axpy_dev<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, which, q * MD_CHUNK, VV, coef, sign, y);
      KCHECK();
    }
  };
  unsigned long long before = g_launches.load();
  CK(cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  try {
    k_copy_indexed<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dV, 0, w.vin.p, 1);      // vin = V[j]
    KCHECK();
    long long dummy = 0;
    precond<T>(w.vin.p, w.zout.p, o, &dummy, u);
    k_copy_indexed<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dZ, 0, w.zout.p, 0);     // Z[j] = zout
    KCHECK();
    kkt_matvec<T>(w.zout.p, w.wst.p, eps, u);
    dots(w.hcol.p);
    axpys(dV, 0, w.hcol.p, -1.0, w.wst.p);
    dots(w.hsum.p);
    axpys(dV, 0, w.hsum.p, -1.0, w.wst.p);
    k_dadd_dev<<<1, 64, 0, st>>>(c, w.hcol.p, w.hsum.p);
    KCHECK();
    flat_dot<T>(st, n, w.wst.p, w.wst.p, w.partial_flat.p, w.scal.p + 2, pm);
    k_givens_dev<<<1, 1, 0, st>>>(c, w.H.p, w.cs.p, w.sn.p, w.g.p, w.hcol.p, w.scal.p + 2, w.scal.p + 3,
                                  w.scal.p + 4);
    KCHECK();
    k_scale_to_indexed<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, c, dV, w.scal.p + 3, w.wst.p);  // V[j+1]
    KCHECK();
    k_fgmres_ctl<<<1, 1, 0, st>>>(c, w.scal.p + 4, h);
    KCHECK();
  } catch (...) {
    cudaGraph_t tmp;
    cudaStreamEndCapture(st, &tmp);
    throw;
  }
  CK(cudaStreamEndCapture(st, &body));
  w.cyc_body_kernels = g_launches.load() - before;
  before = g_launches.load();
  // after the loop: back substitution and x += Z y (k vectors)
  CK(cudaStreamBeginCaptureToGraph(st, g, &wnode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  try {
    k_backsub_dev<<<1, 1, 0, st>>>(c, w.H.p, w.g.p, w.y.p);
    KCHECK();
    axpys(dZ, 1, w.y.p, 1.0, x);
  } catch (...) {
    cudaGraph_t tmp;
    cudaStreamEndCapture(st, &tmp);
    throw;
  }
  CK(cudaStreamEndCapture(st, &g));
  w.cyc_tail_kernels = g_launches.load() - before;
  g_launches.fetch_sub(w.cyc_body_kernels + w.cyc_tail_kernels);   // captured, not launched
  CK(cudaGraphInstantiate(&w.cyc, g, 0));
  w.cyc_key = key;
}

// Right-preconditioned flexible GMRES(m) (Saad 1993) on the KKT matrix, CGS2
// orthogonalisation with FP64 arithmetic on storage of precision T, Givens
// rotations and Hessenberg in FP64 on the device; x = 0 initially.  Sec. 5
// (FSGN-GMRes) and Sec. 6 (30 GMRES iterations per cycle).  Returns 0 when the
// residual estimate reached tol * ||rhs||.
template <typename T>
int Ctx::fgmres(const T *rhs, T *x, double tol, int maxit, double eps, const fwi_opts &o, int *iters,
                long long *inner, const typename cplx<T>::t *u) {
  Work<T> &w = work<T>();
  const int m = w.m;
  const long long n = nkkt;
  T *const *dV = w.dptrV.p;
  T *const *dZ = w.dptrZ.p;
  CK(cudaMemsetAsync(x, 0, n * sizeof(T), st));
  const int pm = o.arnoldi_dots;
  // device control of each restart cycle whenever the preconditioner is
  // graph-replayable (fixed inner iterations); otherwise the host loop below
  const bool devctl = o.use_graph && !(o.inner_tol > 0.0);
  if (devctl) fgmres_cycle_graph<T>(o, eps, x, u);
  flat_dot<T>(st, n, rhs, rhs, w.partial_flat.p, w.scal.p, pm);
  CK(cudaMemcpyAsync(pin, w.scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  const double bnorm = std::sqrt(pin[0]);
  if (!(bnorm > 0.0)) return 0;
  if (!std::isfinite(bnorm)) fail(FWI_E_NUMERIC, "non-finite right-hand side in FGMRES");
  const T *r = rhs;
  double beta = bnorm;
  int total = 0;
  bool conv = false;
  // loss of orthogonality of a cycle's basis V_0 .. V_k: max |delta_ij - V_i . V_j|
  // (FP64 products; diagnostics only, one multi-dot per basis vector)
  auto orth_check = [&](int k) {
    if (k <= 0) return;
    std::vector<double> hh(k + 1);
    for (int jj = 0; jj <= k; ++jj) {
      multidot<T>(n, jj + 1, dV, w.V.p + (size_t)jj * w.ld, w.hsum.p, 0, DOT_FP64);
      CK(cudaMemcpyAsync(hh.data(), w.hsum.p, (jj + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
      sync();
      for (int ii = 0; ii <= jj; ++ii) orth_loss = std::max(orth_loss, std::fabs((ii == jj ? 1.0 : 0.0) - hh[ii]));
    }
  };
  while (total < maxit && !conv) {
    CK(cudaMemcpyAsync(w.scal.p + 1, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
    KPROF("k_scale_inv", -1, 2.0 * n * sizeof(T), st);
    k_scale_inv<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, w.scal.p + 1, r, w.V.p);
    KCHECK();
    std::vector<double> g0(m + 1, 0.0);
    g0[0] = beta;
    CK(cudaMemcpyAsync(w.g.p, g0.data(), (m + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
    if (devctl) {
      // the whole cycle on the device; the host reads the control block once
      FgCtl *hc = reinterpret_cast<FgCtl *>(pin);
      hc->j = 0; hc->k = 0; hc->total = total; hc->state = 0; hc->m = m; hc->maxit = maxit;
      hc->thr = tol * bnorm;
      CK(cudaMemcpyAsync(w.ctl.p, hc, sizeof(FgCtl), cudaMemcpyHostToDevice, st));
      CK(cudaGraphLaunch(w.cyc, st));
      CK(cudaMemcpyAsync(hc, w.ctl.p, sizeof(FgCtl), cudaMemcpyDeviceToHost, st));
      sync();
      const int kk = hc->k;
      g_launches.fetch_add(w.cyc_body_kernels * (unsigned long long)kk + w.cyc_tail_kernels);
      if (inner && o.inner_solver != 2) *inner += 2LL * o.inner_iters * B * kk;
      total = hc->total;
      const int state = hc->state;
      if (state == 2) fail(FWI_E_NUMERIC, "non-finite residual in FGMRES");
      if (state == 1) conv = true;
      if (o.check_orth) orth_check(kk);
      if (conv || total >= maxit) break;
    } else {
    int k = 0;
    for (int j = 0; j < m && total < maxit; ++j) {
      T *vj = w.V.p + (size_t)j * w.ld;
      T *zj = w.Z.p + (size_t)j * w.ld;
      T *wv = w.V.p + (size_t)(j + 1) * w.ld;
      precond_any<T>(vj, zj, o, inner, u);
      kkt_matvec<T>(zj, wv, eps, u);
      // classical Gram-Schmidt, twice
      multidot<T>(n, j + 1, dV, wv, w.hcol.p, 0, pm);
      multi_axpy<T>(n, j + 1, dV, w.hcol.p, -1.0, wv);
      multidot<T>(n, j + 1, dV, wv, w.hsum.p, 0, pm);
      multi_axpy<T>(n, j + 1, dV, w.hsum.p, -1.0, wv);
      KPROF("k_dadd", -1, 0, st);
      k_dadd<<<1, 64, 0, st>>>(j + 1, w.hcol.p, w.hsum.p);
      KCHECK();
      flat_dot<T>(st, n, wv, wv, w.partial_flat.p, w.scal.p + 2, pm);
      KPROF("k_givens", -1, 0, st);
      k_givens<<<1, 1, 0, st>>>(j, m, w.H.p, w.cs.p, w.sn.p, w.g.p, w.hcol.p, w.scal.p + 2, w.scal.p + 3,
                                w.scal.p + 4);
      KCHECK();
      KPROF("k_scale_inv", -1, 2.0 * n * sizeof(T), st);
      k_scale_inv<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, w.scal.p + 3, wv, wv);
      KCHECK();
      CK(cudaMemcpyAsync(pin, w.scal.p + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
      sync();
      ++total;
      k = j + 1;
      if (!std::isfinite(pin[0])) fail(FWI_E_NUMERIC, "non-finite residual in FGMRES");
      if (pin[0] / bnorm <= tol) { conv = true; break; }
    }
    if (o.check_orth) orth_check(k);
    KPROF("k_backsub", -1, 0, st);
    k_backsub<<<1, 1, 0, st>>>(k, m, w.H.p, w.g.p, w.y.p);
    KCHECK();
    multi_axpy<T>(n, k, dZ, w.y.p, 1.0, x);
    if (conv || total >= maxit) break;
    }
    // restart from r = rhs - M x
    kkt_matvec<T>(x, w.tmp.p, eps, u);
    KPROF("k_axpby", -1, 3.0 * n * sizeof(T), st);
    k_axpby<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, 1.0, rhs, -1.0, w.tmp.p);
    KCHECK();
    r = w.tmp.p;
    flat_dot<T>(st, n, r, r, w.partial_flat.p, w.scal.p, pm);
    CK(cudaMemcpyAsync(pin, w.scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    beta = std::sqrt(pin[0]);
    if (beta / bnorm <= tol) { conv = true; break; }
  }
  if (iters) *iters += total;
  return conv ? 0 : 1;
}


// Outer BiCGStab (van der Vorst 1992) on the KKT matrix in the real inner
// product, right-preconditioned by the block-triangular preconditioner: the
// memory-lean alternative to FGMRES named in the paper's conclusions (eight
// KKT-size vectors instead of 2m + 1).  Two preconditioner applications and two
// KKT products per iteration; x = 0 initially; stops when the recursively
// updated residual reaches tol * ||rhs|| (the caller's FP64 refinement checks
// the true residual).  Returns 0 when converged.
template <typename T>
int Ctx::bicgstab_outer(const T *rhs, T *x, double tol, int maxit, double eps, const fwi_opts &o, int *iters,
                        long long *inner, const typename cplx<T>::t *u) {
  Work<T> &w = work<T>();
  const long long n = nkkt;
  for (auto &v : w.ob) v.alloc(n);
  T *r = w.ob[0].p, *rh = w.ob[1].p, *p = w.ob[2].p, *v = w.ob[3].p, *sv = w.ob[4].p, *t = w.ob[5].p,
    *ph = w.ob[6].p, *sh = w.ob[7].p;
  const int pm = o.arnoldi_dots;
  auto dot = [&](const T *a, const T *b) {
    flat_dot<T>(st, n, a, b, w.partial_flat.p, w.scal.p, pm);
    CK(cudaMemcpyAsync(pin, w.scal.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    return pin[0];
  };
  auto axpby = [&](double a, const T *xx, double b, T *yy) {   // yy = a xx + b yy
    KPROF("k_axpby", -1, 3.0 * n * sizeof(T), st);
    k_axpby<T><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(n, a, xx, b, yy);
    KCHECK();
  };
  CK(cudaMemsetAsync(x, 0, n * sizeof(T), st));
  CK(cudaMemcpyAsync(r, rhs, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(rh, rhs, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemsetAsync(p, 0, n * sizeof(T), st));
  CK(cudaMemsetAsync(v, 0, n * sizeof(T), st));
  const double bnorm = std::sqrt(dot(rhs, rhs));
  if (!(bnorm > 0.0)) return 0;
  if (!std::isfinite(bnorm)) fail(FWI_E_NUMERIC, "non-finite right-hand side in BiCGStab");
  double rho = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  bool conv = false;
  while (it < maxit) {
    const double rho_new = dot(rh, r);
    if (rho_new == 0.0 || !std::isfinite(rho_new)) break;
    const double beta = it == 0 ? 0.0 : (rho_new / rho) * (alpha / omega);
    axpby(-omega, v, 1.0, p);                 // p = p - omega v
    axpby(1.0, r, beta, p);                   // p = r + beta p
    precond_any<T>(p, ph, o, inner, u);       // ph = P~^{-1} p
    kkt_matvec<T>(ph, v, eps, u);             // v = M ph
    const double rv = dot(rh, v);
    if (rv == 0.0 || !std::isfinite(rv)) break;
    alpha = rho_new / rv;
    CK(cudaMemcpyAsync(sv, r, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    axpby(-alpha, v, 1.0, sv);                // s = r - alpha v
    precond_any<T>(sv, sh, o, inner, u);      // sh = P~^{-1} s
    kkt_matvec<T>(sh, t, eps, u);             // t = M sh
    const double tt = dot(t, t);
    omega = tt > 0.0 ? dot(t, sv) / tt : 0.0;
    axpby(alpha, ph, 1.0, x);                 // x += alpha ph + omega sh
    axpby(omega, sh, 1.0, x);
    CK(cudaMemcpyAsync(r, sv, n * sizeof(T), cudaMemcpyDeviceToDevice, st));
    axpby(-omega, t, 1.0, r);                 // r = s - omega t
    rho = rho_new;
    ++it;
    const double rn = std::sqrt(dot(r, r));
    if (!std::isfinite(rn)) fail(FWI_E_NUMERIC, "non-finite residual in BiCGStab");
    if (rn <= tol * bnorm) { conv = true; break; }
    if (omega == 0.0) break;
  }
  if (iters) *iters += it;
  return conv ? 0 : 1;
}

template <> const float2 *Ctx::u_T<float>() {
  if (u_version32 != fwd_version) {
    KPROF("k_convert", 0, 12.0 * 2 * F0, st);
    k_convert<double, float><<<grid_for(2 * F0, 256), 256, 0, st>>>(2 * F0, (const double *)u64.p, (float *)w32.u.p);
    KCHECK();
    u_version32 = fwd_version;
  }
  return w32.u.p;
}
template <> const double2 *Ctx::u_T<double>() { return u64.p; }

// Per-block FP64-refined solve of A' x = rhs (cj = 1: A'^H): inner solves in
// precision T on the normalised residual, update and residual in FP64, until
// every block satisfies ||rhs - A' x|| <= fwd_tol ||rhs|| (Sec. 2, Au = f).
template <typename T>
int Ctx::refined_solve(const double2 *rhs, double2 *x, int cj, const fwi_opts &o, fwi_stats *stats, bool warm) {
  typedef typename cplx<T>::t T2;
  ensure_work<T>(o);
  Work<T> &w = work<T>();
  LevelView<double> L64 = viewA<double>();
  LevelView<T> LT = viewA<T>();
  const int nt = L64.n_tiles;
  rho64.alloc(F0);
  if (warm) {
    // start from the wavefields x already holds: rho = rhs - A' x in FP64
    field_op<double>(FM_RESID, cj, 0.0, x, rhs, rho64.p, true, 0);
  } else {
    CK(cudaMemsetAsync(x, 0, F0 * sizeof(double2), st));
    CK(cudaMemcpyAsync(rho64.p, rhs, F0 * sizeof(double2), cudaMemcpyDeviceToDevice, st));
  }
  std::vector<double> n0(B), nb(B), fac(B);
  auto block_norms = [&](const double2 *v, std::vector<double> &out) {
    block_dots<double>(1, v, v, nullptr, nullptr, nullptr, nullptr);
    std::vector<double2> hp((size_t)nt * 3);
    CK(cudaMemcpyAsync(hp.data(), partial.p, hp.size() * sizeof(double2), cudaMemcpyDeviceToHost, st));
    sync();
    for (int b = 0; b < B; ++b) {
      double a = 0.0;
      for (int t = lv[0].ht0[b]; t < lv[0].ht1[b]; ++t) a += hp[(size_t)t * 3].x;
      out[b] = std::sqrt(a);
    }
  };
  block_norms(rhs, n0);
  int sweeps = 0;
  int status = FWI_E_NOCONV;
  T2 *rT = (T2 *)w.vin.p;
  T2 *eT = (T2 *)w.zout.p;
  const double inner_tol = sizeof(T) == 4 ? 1e-5 : std::max(o.fwd_tol * 0.1, 1e-15);
  // iterations per sweep: start at fwd_iters; a sweep that reduced the worst
  // unconverged block by less than 20x doubles it (up to 8 x fwd_iters)
  int iters = o.fwd_iters;
  std::vector<double> prev(B, 0.0);
  for (;;) {
    block_norms(rho64.p, nb);
    double worst = 0.0, slow = 0.0;
    bool finite = true;
    for (int b = 0; b < B; ++b) {
      if (!std::isfinite(nb[b])) finite = false;
      if (n0[b] > 0.0) {
        double rel = nb[b] / n0[b];
        worst = std::max(worst, rel);
        if (sweeps > 0 && rel > o.fwd_tol && prev[b] > 0.0) slow = std::max(slow, nb[b] / prev[b]);
      }
    }
    if (!finite) fail(FWI_E_NUMERIC, "non-finite residual in the forward/adjoint solve");
    if (stats) stats->fwd_rel_res = worst;
    if (worst <= o.fwd_tol) { status = FWI_OK; break; }
    if (sweeps >= o.max_fwd_refine) break;
    if (slow > 0.05) iters = std::min(2 * iters, 8 * o.fwd_iters);
    prev = nb;
    for (int b = 0; b < B; ++b) fac[b] = nb[b] > 0.0 ? 1.0 / nb[b] : 0.0;
    CK(cudaMemcpyAsync(blkfac.p, fac.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
    KPROF("k_blk_scale", 0, (16.0 + sizeof(typename cplx<T>::t)) * F0, st);
    k_blk_scale<double, T, T><<<nt, TILE_THREADS, 0, st>>>(LT, (const double *)rho64.p, blkfac.p, (T *)rT, 0);
    KCHECK();
    long long cnt = 0;
    inner_solve<T>(rT, eT, cj, iters, inner_tol, o, &cnt);
    if (stats) stats->inner_iters += cnt;
    CK(cudaMemcpyAsync(blkfac.p, nb.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
    KPROF("k_blk_scale", 0, (sizeof(typename cplx<T>::t) + 32.0) * F0, st);
    k_blk_scale<T, double, T><<<nt, TILE_THREADS, 0, st>>>(LT, (const T *)eT, blkfac.p, (double *)x, 1);
    KCHECK();
    field_op<double>(FM_RESID, cj, 0.0, x, rhs, rho64.p, true, 0);
    ++sweeps;
  }
  if (stats) stats->fwd_sweeps += sweeps;
  return status;
}

// a2 + a3: forward wavefields of every block, predicted data, residuals, misfit.
void Ctx::forward(const fwi_opts &o, fwi_stats *stats) {
  build_hierarchy(o);
  auto t0 = std::chrono::steady_clock::now();
  u64.alloc(F0);
  f64.alloc(F0);
  f64.zero(st);
  KPROF("k_set_sources", -1, 0, st);
  k_set_sources<<<grid_for(B, 128), 128, 0, st>>>(B, d_src_node.p, d_src_amp.p, f64.p);
  KCHECK();
  // warm start from the previous forward wavefields of this layout (a Newton
  // trajectory changes the model a little per step); same fwd_tol either way
  const bool warm = o.fwd_warm && u64_valid && u64.n == (size_t)F0;
  u64_valid = false;
  int rc = o.precision == FWI_C128 ? refined_solve<double>(f64.p, u64.p, 0, o, stats, warm)
                                   : refined_solve<float>(f64.p, u64.p, 0, o, stats, warm);
  u64_valid = rc == FWI_OK;
  if (stats) stats->fwd_warm = warm ? 1 : 0;
  ++fwd_version;
  // receivers: q = Q u, r = d - q
  int nrec = (int)rec_node.size();
  q.alloc(std::max(1, nrec));
  r.alloc(std::max(1, nrec));
  bool have_d = true;
  for (auto &I : inst) have_d = have_d && I.has_data;
  DBuf<double2> dd;
  if (have_d && nrec) {
    // observed data in receiver-entry order (blocks in order; per block the
    // source's receivers at the block's frequency): one copy per block
    dd.alloc(nrec);
    int e = 0;
    for (int b = 0; b < B; ++b) {
      Instance &I = inst[blk_inst[b]];
      int k = blk_src[b], f = blk_freq[b];
      int cnt = I.rec_off[k + 1] - I.rec_off[k];
      if (cnt)
        CK(cudaMemcpyAsync(dd.p + e, I.d.p + (long long)f * I.rec_total() + I.rec_off[k], cnt * sizeof(double2),
                           cudaMemcpyDeviceToDevice, st));
      e += cnt;
    }
  }
  if (nrec) {
    KPROF("k_rec_residual", -1, 0, st);
    k_rec_residual<<<grid_for(nrec, 128, 1 << 20), 128, 0, st>>>(nrec, d_rec_node.p, u64.p, have_d ? dd.p : nullptr,
                                                                 q.p, r.p, have_d ? 1 : 0);
    KCHECK();
  }
  // misfit per instance
  std::vector<int> e0(inst.size()), e1(inst.size());
  {
    int e = 0;
    for (size_t i = 0; i < inst.size(); ++i) {
      e0[i] = e;
      for (int b = h_inst[i].blk0; b < h_inst[i].blk1; ++b) {
        Instance &I = inst[i];
        e += I.rec_off[blk_src[b] + 1] - I.rec_off[blk_src[b]];
      }
      e1[i] = e;
    }
  }
  DBuf<int> de0, de1;
  de0.upload(e0, st);
  de1.upload(e1, st);
  misfit_d.alloc(inst.size());
  KPROF("k_misfit", -1, 0, st);
  k_misfit<<<(int)inst.size(), 256, 0, st>>>(de0.p, de1.p, d_rec_w.p, r.p, misfit_d.p);
  KCHECK();
  misfit.assign(inst.size(), 0.0);
  CK(cudaMemcpyAsync(misfit.data(), misfit_d.p, inst.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  have_fwd = true;
  if (stats) {
    stats->t_forward_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    double m = 0.0;
    for (double v : misfit) m += v;
    stats->misfit = m;
  }
  if (rc != FWI_OK) fail(FWI_E_NOCONV, "forward solve did not reach fwd_tol within max_fwd_refine sweeps");
}

// per-instance ||x||^2 of a packed FP64 vector -> host vector
void Ctx::seg_norms(const double *x) {
  const int nb = 64;
  dim3 g(nb, (unsigned)h_segs.size());
  KPROF("k_seg_norm2", -1, 8.0 * nkkt, st);
  k_seg_norm2<double><<<g, FLAT_THREADS, 0, st>>>(d_segs.p, x, seg_partial.p, nb);
  KCHECK();
}

// ds (all instances' cores) = fac_i * (ctrl part of a packed FP64 vector)
void Ctx::write_ctrl(const double *src_ctrl_dev, double *dst, int on_device, const double *fac) {
  std::vector<SegDev> cs;
  for (size_t i = 0; i < inst.size(); ++i)
    cs.push_back(SegDev{h_inst[i].ctrl, h_inst[i].ctrl + (long long)inst[i].g.nx * inst[i].g.nz, (int)i});
  DBuf<SegDev> dcs;
  dcs.upload(cs, st);
  DBuf<double> f, out;
  std::vector<double> hf(fac, fac + inst.size());
  f.upload(hf, st);
  double *target = dst;
  if (!on_device) { out.alloc(Nc); target = out.p; }
  KPROF("k_seg_scale", -1, 16.0 * Nc, st);
  k_seg_scale<double, double><<<dim3(64, (unsigned)cs.size()), 256, 0, st>>>(dcs.p, src_ctrl_dev, f.p, target);
  KCHECK();
  if (!on_device) CK(cudaMemcpyAsync(dst, out.p, Nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
}

// a4-a8: the KKT solve with the block-triangular preconditioner, FGMRES and FP64 refinement.
int Ctx::kkt_solve(const fwi_opts &o, fwi_stats *stats) {
  if (!have_fwd) fail(FWI_E_INVAL, "fwi_kkt_solve needs fwi_forward at the current model");
  bool have_d = true;
  for (auto &I : inst) have_d = have_d && I.has_data;
  if (!have_d) fail(FWI_E_INVAL, "observed data missing");
  if (!(o.eps > 0.0)) fail(FWI_E_INVAL, "eps must be > 0");
  auto t0 = std::chrono::steady_clock::now();
  b64.alloc(nkkt); xi64.alloc(nkkt); rho_k64.alloc(nkkt);
  b64.zero(st);
  // b_u = Q^T W^T W r (FP64 field in the du slot)
  int nrec = (int)rec_node.size();
  if (n_unique) {
    KPROF("k_rec_scatter", -1, 0, st);
    k_rec_scatter<<<grid_for(n_unique, 128, 1 << 20), 128, 0, st>>>(n_unique, d_unode.p, d_uoff.p, d_uidx.p, d_rec_w.p,
                                                                    r.p, (double2 *)b64.p);
  }
  KCHECK();
  (void)nrec;
  {
    std::vector<const double *> sp;
    std::vector<double> gr;
    for (auto &I : inst) { sp.push_back(I.s.p); gr.push_back(I.gamma_ref); }
    DBuf<const double *> dsp;
    dsp.upload(sp, st);
    inst_gref.upload(gr, st);
    long long mx = 0;
    for (auto &I : inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
    KPROF("k_ctrl_rhs", -1, 0, st);
    k_ctrl_rhs<<<dim3(grid_for(mx, 256), (unsigned)inst.size()), 256, 0, st>>>(d_inst.p, dsp.p, inst_gref.p, o.eps,
                                                                              o.include_Ls_n, b64.p + 4 * F0);
    KCHECK();
    sync();
  }
  const int n_inst = (int)inst.size();
  auto inst_norms = [&](const double *x, std::vector<double> &out) {
    seg_norms(x);
    std::vector<double> hp(h_segs.size() * 64);
    CK(cudaMemcpyAsync(hp.data(), seg_partial.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    sync();
    out.assign(n_inst, 0.0);
    for (size_t sgi = 0; sgi < h_segs.size(); ++sgi)
      for (int q2 = 0; q2 < 64; ++q2) out[h_segs[sgi].inst] += hp[sgi * 64 + q2];
    for (auto &v : out) v = std::sqrt(v);
  };
  std::vector<double> bn, rn;
  inst_norms(b64.p, bn);
  CK(cudaMemsetAsync(xi64.p, 0, nkkt * sizeof(double), st));
  CK(cudaMemcpyAsync(rho_k64.p, b64.p, nkkt * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const bool c128 = o.precision == FWI_C128;
  if (o.inner_solver >= 1) ensure_ilu();     // before any graph capture
  hblock_prepare(o);
  if (o.outer_solver == 1) {
    // the outer BiCGStab allocates its eight vectors itself (no Krylov basis)
    if (c128) ensure_work<double>(o); else ensure_work<float>(o);
  } else {
    if (c128) ensure_krylov<double>(o); else ensure_krylov<float>(o);
  }
  int outer = 0, sweeps = 0;
  long long inner = 0;
  double worst = 0.0;
  int status = FWI_E_NOCONV;
  orth_loss = 0.0;
  for (;;) {
    inst_norms(rho_k64.p, rn);
    worst = 0.0;
    for (int i = 0; i < n_inst; ++i) {
      if (!std::isfinite(rn[i])) fail(FWI_E_NUMERIC, "non-finite KKT residual");
      if (bn[i] > 0.0) worst = std::max(worst, rn[i] / bn[i]);
    }
    if (worst <= o.tol) { status = FWI_OK; break; }
    if (sweeps >= o.max_refine || outer >= o.max_outer) break;
    std::vector<double> fac(n_inst), back(n_inst);
    for (int i = 0; i < n_inst; ++i) {
      fac[i] = rn[i] > 0.0 ? 1.0 / rn[i] : 0.0;
      back[i] = rn[i];
    }
    inst_fac.upload(fac, st);
    dim3 g(64, (unsigned)h_segs.size());
    int left = o.max_outer - outer;
    if (c128) {
      Work<double> &w = w64;
      KPROF("k_seg_scale", -1, 16.0 * nkkt, st);
      k_seg_scale<double, double><<<g, 256, 0, st>>>(d_segs.p, rho_k64.p, inst_fac.p, w.rhs.p);
      KCHECK();
      if (o.outer_solver == 1)
        bicgstab_outer<double>(w.rhs.p, w.sol.p, std::max(o.tol * 0.5, 1e-14), left, o.eps, o, &outer, &inner,
                               u_T<double>());
      else
        fgmres<double>(w.rhs.p, w.sol.p, std::max(o.tol * 0.5, 1e-14), left, o.eps, o, &outer, &inner, u_T<double>());
      inst_fac.upload(back, st);
      KPROF("k_seg_axpy", -1, 24.0 * nkkt, st);
      k_seg_axpy<double><<<g, 256, 0, st>>>(d_segs.p, w.sol.p, inst_fac.p, xi64.p);
      KCHECK();
    } else {
      Work<float> &w = w32;
      KPROF("k_seg_scale", -1, 12.0 * nkkt, st);
      k_seg_scale<double, float><<<g, 256, 0, st>>>(d_segs.p, rho_k64.p, inst_fac.p, w.rhs.p);
      KCHECK();
      if (o.outer_solver == 1)
        bicgstab_outer<float>(w.rhs.p, w.sol.p, o.sweep_tol, left, o.eps, o, &outer, &inner, u_T<float>());
      else
        fgmres<float>(w.rhs.p, w.sol.p, o.sweep_tol, left, o.eps, o, &outer, &inner, u_T<float>());
      inst_fac.upload(back, st);
      KPROF("k_seg_axpy", -1, 20.0 * nkkt, st);
      k_seg_axpy<float><<<g, 256, 0, st>>>(d_segs.p, w.sol.p, inst_fac.p, xi64.p);
      KCHECK();
    }
    // rho = b - M xi in FP64 (c128 matvec with the FP64 wavefields)
    kkt_matvec<double>(xi64.p, rho_k64.p, o.eps, u64.p);
    KPROF("k_axpby", -1, 24.0 * nkkt, st);
    k_axpby<double><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(nkkt, 1.0, b64.p, -1.0, rho_k64.p);
    KCHECK();
    ++sweeps;
  }
  if (stats) {
    stats->outer_iters += outer;
    stats->refinements += sweeps;
    stats->inner_iters += inner;
    stats->rel_res = worst;
    stats->orth_loss = orth_loss;
    stats->t_solve_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return status;
}

int Ctx::gradient(const fwi_opts &o, double *misfit_out, double *grad, int on_device, fwi_stats *stats) {
  forward(o, stats);
  bool have_d = true;
  for (auto &I : inst) have_d = have_d && I.has_data;
  if (!have_d) fail(FWI_E_INVAL, "observed data missing");
  // adjoint right-hand side Q^T W^T W r and lambda' = A'^{-H} rhs
  DBuf<double2> rhs, lam;
  rhs.alloc(F0); lam.alloc(F0);
  rhs.zero(st);
  if (n_unique) {
    KPROF("k_rec_scatter", -1, 0, st);
    k_rec_scatter<<<grid_for(n_unique, 128, 1 << 20), 128, 0, st>>>(n_unique, d_unode.p, d_uoff.p, d_uidx.p, d_rec_w.p,
                                                                    r.p, rhs.p);
  }
  KCHECK();
  int rc = o.precision == FWI_C128 ? refined_solve<double>(rhs.p, lam.p, 1, o, stats)
                                   : refined_solve<float>(rhs.p, lam.p, 1, o, stats);
  DBuf<double> g;
  double *target = grad;
  if (!on_device) { g.alloc(Nc); target = g.p; }
  long long mx = 0;
  for (auto &I : inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
  dim3 gr((unsigned)((mx + 127) / 128), (unsigned)inst.size());
  KPROF("k_coupling_reduce", 2, 32.0 * cpl_nodes() + 8.0 * Nc, st);
  k_coupling_reduce<double, double><<<gr, dim3(128, CPL_ROWS), 0, st>>>(d_inst.p, d_blk_off.p, cfG.p, u64.p,
                                                                 lam.p, nullptr, 0.0, 2, target);
  KCHECK();
  if (!on_device) CK(cudaMemcpyAsync(grad, g.p, Nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  if (misfit_out)
    for (size_t i = 0; i < inst.size(); ++i) misfit_out[i] = misfit[i];
  if (rc != FWI_OK) fail(FWI_E_NOCONV, "adjoint solve did not reach fwd_tol");
  return FWI_OK;
}

int Ctx::newton_step(const fwi_opts &o, double *ds, int on_device, fwi_stats *stats) {
  auto t0 = std::chrono::steady_clock::now();
  build_hierarchy(o);
  if (stats) stats->t_setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  forward(o, stats);
  int rc = kkt_solve(o, stats);
  apply_update(ds, on_device);
  return rc;
}

// The update of a Gauss-Newton step from the scaled control in xi64's ds slot.
void Ctx::apply_update(double *ds, int on_device) {
  // ds = gamma_ref * ds~ ; s += ds
  std::vector<double> gr;
  for (auto &I : inst) gr.push_back(I.gamma_ref);
  DBuf<double> dsd;
  dsd.alloc(Nc);
  write_ctrl(xi64.p + 4 * F0, dsd.p, 1, gr.data());
  std::vector<double *> sp;
  for (auto &I : inst) sp.push_back(I.s.p);
  DBuf<double *> dsp;
  dsp.upload(sp, st);
  long long mx = 0;
  for (auto &I : inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
  KPROF("k_update_model", -1, 0, st);
  k_update_model<<<dim3(grid_for(mx, 256), (unsigned)inst.size()), 256, 0, st>>>(d_inst.p, dsp.p, dsd.p);
  KCHECK();
  if (ds) {
    if (on_device) CK(cudaMemcpyAsync(ds, dsd.p, Nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else CK(cudaMemcpyAsync(ds, dsd.p, Nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  sync();
  ++model_version;
  have_fwd = false;
}

// The matrix-free Gauss-Newton normal operator of the scaled control (Sec. 3,
// eq. normal_system_discrete_sum):
//   H~ v = eps v + Re(P~^H A'^{-H} F A'^{-1} P~ v),  F = Q^T W^T W Q,
// one forward and one adjoint FP64-refined block solve of every block per
// product (complex64 or complex128 inner solves, opts.fwd_tol), and the
// right-hand side of the normal equations.  Used by RSGN-CG and by the
// power iteration for the largest eigenvalue of Re(J~^H W^T W J~).
struct NormalOp {
  Ctx &c;
  const fwi_opts &o;
  fwi_stats *stats;
  long long nc;
  dim3 gr;
  DBuf<double2> fa, fb, zero, qv, rdummy;
  DBuf<double> part;
  int solve_rc = FWI_OK;
  NormalOp(Ctx &cc, const fwi_opts &oo, fwi_stats *ss) : c(cc), o(oo), stats(ss), nc(cc.Nc) {
    fa.alloc(c.F0); fb.alloc(c.F0); zero.alloc(c.F0);
    zero.zero(c.st);
    part.alloc(FLAT_BLOCKS);
    const int nrec = (int)c.rec_node.size();
    qv.alloc(std::max(nrec, 1)); rdummy.alloc(std::max(nrec, 1));
    long long mx = 0;
    for (auto &I : c.inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
    gr = dim3((unsigned)((mx + 127) / 128), (unsigned)c.inst.size());
  }
  void solve(const double2 *rhs, double2 *sol, int cj) {
    int rc = o.precision == FWI_C128 ? c.refined_solve<double>(rhs, sol, cj, o, stats)
                                     : c.refined_solve<float>(rhs, sol, cj, o, stats);
    if (rc != FWI_OK) solve_rc = rc;
  }
  // out = eps * v + Re(P~^H lambda)  (per core node, fixed block order)
  void couple(const double2 *lam, const double *v, double eps, double *out) {
    cudaStream_t st = c.st;
    KPROF("k_coupling_reduce", 3, 32.0 * c.cpl_nodes() + 16.0 * c.Nc, st);
    k_coupling_reduce<double, double><<<gr, dim3(128, CPL_ROWS), 0, st>>>(c.d_inst.p, c.d_blk_off.p, c.cfK.p,
                                                                        c.u64.p, lam, v, eps, 3, out);
    KCHECK();
  }
  // lambda = A'^{-H} Q^T W^T W (values at the receivers q)
  void adjoint_of_receivers(const double2 *q, double2 *lam) {
    cudaStream_t st = c.st;
    CK(cudaMemsetAsync(fa.p, 0, c.F0 * sizeof(double2), st));
    if (c.n_unique) {
      KPROF("k_rec_scatter", -1, 0, st);
      k_rec_scatter<<<grid_for(c.n_unique, 128, 1 << 20), 128, 0, st>>>(c.n_unique, c.d_unode.p, c.d_uoff.p,
                                                                        c.d_uidx.p, c.d_rec_w.p, q, fa.p);
    }
    KCHECK();
    solve(fa.p, lam, 1);
  }
  // out = H~ v (eps = o.eps) or the Gauss-Newton part alone (eps = 0)
  void apply(const double *v, double eps, double *out) {
    cudaStream_t st = c.st;
    LevelView<double> L64 = c.viewA<double>();
    KPROF("k_coupling_scatter", 0, 48.0 * c.F0, st);
    k_coupling_scatter<double><<<L64.n_tiles, TILE_THREADS, 0, st>>>(L64, c.d_inst.p, c.cfK.p, c.u64.p, zero.p, v,
                                                                     fb.p);
    KCHECK();
    solve(fb.p, fa.p, 0);                                  // du = A'^{-1} P~ v
    const int nrec = (int)c.rec_node.size();
    if (nrec) {
      KPROF("k_rec_residual", -1, 0, st);
      k_rec_residual<<<grid_for(nrec, 128, 1 << 20), 128, 0, st>>>(nrec, c.d_rec_node.p, fa.p, nullptr, qv.p,
                                                                   rdummy.p, 0);
    }
    KCHECK();
    adjoint_of_receivers(qv.p, fb.p);                      // lambda = A'^{-H} F du
    couple(fb.p, v, eps, out);
  }
  double dot(const double *a, const double *b) {
    KPROF("k_dot2", -1, 16.0 * nc, c.st);
    k_dot2<double><<<FLAT_BLOCKS, FLAT_THREADS, 0, c.st>>>(nc, a, b, part.p);
    KCHECK();
    std::vector<double> h(FLAT_BLOCKS);
    CK(cudaMemcpyAsync(h.data(), part.p, FLAT_BLOCKS * sizeof(double), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    double acc = 0.0;
    for (double v : h) acc += v;
    return acc;
  }
};

// Reduced-space Gauss-Newton (Sec. 3, eq. normal_system_discrete_sum) by
// conjugate gradients, on the same scaled variables as the KKT solve:
//   (eps I + Re(P~^H A'^{-H} F A'^{-1} P~)) ds~ = b_s + Re(P~^H A'^{-H} Q^T W^T W r),
// F = Q^T W^T W Q, which is the KKT system with du and lambda eliminated, so
// its solution is the KKT solution's ds~.  Every CG iteration makes one
// forward and one adjoint refined solve of every block (FP64 fields, complex64
// inner solves, fwd_tol).  The result goes to xi64's ds slot; stats->outer_iters
// counts CG iterations, stats->rel_res is the final ||g - H ds~|| / ||g||
// (the recursively updated CG residual).
int Ctx::rsgn_solve(const fwi_opts &o, fwi_stats *stats) {
  if (!have_fwd) fail(FWI_E_INVAL, "the reduced-space step needs fwi_forward at the current model");
  bool have_d = true;
  for (auto &I : inst) have_d = have_d && I.has_data;
  if (!have_d) fail(FWI_E_INVAL, "observed data missing");
  if (!(o.eps > 0.0)) fail(FWI_E_INVAL, "eps must be > 0");
  auto t0 = std::chrono::steady_clock::now();
  const long long nc = Nc;
  xi64.alloc(nkkt);
  CK(cudaMemsetAsync(xi64.p, 0, nkkt * sizeof(double), st));
  double *x = xi64.p + 4 * F0;             // ds~ (the KKT layout's control slot)
  DBuf<double> g, rr, p, hp, bs;
  g.alloc(nc); rr.alloc(nc); p.alloc(nc); hp.alloc(nc); bs.alloc(nc);
  NormalOp N(*this, o, stats);
  long long mx = 0;
  for (auto &I : inst) mx = std::max(mx, (long long)I.g.nx * I.g.nz);
  // right-hand side g = b_s + Re(P~^H A'^{-H} Q^T W^T W r)
  {
    std::vector<const double *> sp;
    std::vector<double> gref;
    for (auto &I : inst) { sp.push_back(I.s.p); gref.push_back(I.gamma_ref); }
    DBuf<const double *> dsp;
    dsp.upload(sp, st);
    inst_gref.upload(gref, st);
    DBuf<double> bsfull;
    bsfull.alloc(nkkt);
    KPROF("k_ctrl_rhs", -1, 0, st);
    k_ctrl_rhs<<<dim3(grid_for(mx, 256), (unsigned)inst.size()), 256, 0, st>>>(d_inst.p, dsp.p, inst_gref.p, o.eps,
                                                                              o.include_Ls_n, bsfull.p + 4 * F0);
    KCHECK();
    CK(cudaMemcpyAsync(bs.p, bsfull.p + 4 * F0, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
    N.adjoint_of_receivers(r.p, N.fb.p);
    N.couple(N.fb.p, bs.p, 1.0, g.p);
    sync();
  }
  // CG from ds~ = 0
  CK(cudaMemcpyAsync(rr.p, g.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(p.p, g.p, nc * sizeof(double), cudaMemcpyDeviceToDevice, st));
  const double gn = std::sqrt(N.dot(g.p, g.p));
  double rho = gn * gn;
  int it = 0;
  int status = FWI_E_NOCONV;
  double rel = gn > 0.0 ? 1.0 : 0.0;
  if (!(gn > 0.0)) status = FWI_OK;
  while (status != FWI_OK && it < o.max_outer) {
    N.apply(p.p, o.eps, hp.p);
    const double php = N.dot(p.p, hp.p);
    if (!std::isfinite(php) || !(php > 0.0)) fail(FWI_E_NUMERIC, "reduced-space CG: p^T H p is not positive");
    const double alpha = rho / php;
    KPROF("k_axpby", -1, 24.0 * nc, st);
    k_axpby<double><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(nc, alpha, p.p, 1.0, x);
    KCHECK();
    KPROF("k_axpby", -1, 24.0 * nc, st);
    k_axpby<double><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(nc, -alpha, hp.p, 1.0, rr.p);
    KCHECK();
    const double rho_new = N.dot(rr.p, rr.p);
    ++it;
    rel = std::sqrt(rho_new) / gn;
    if (rel <= o.tol) { status = FWI_OK; break; }
    KPROF("k_axpby", -1, 24.0 * nc, st);
    k_axpby<double><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(nc, 1.0, rr.p, rho_new / rho, p.p);
    KCHECK();
    rho = rho_new;
  }
  sync();
  if (stats) {
    stats->outer_iters += it;
    stats->rel_res = rel;
    stats->t_solve_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  if (N.solve_rc != FWI_OK && status == FWI_OK) status = N.solve_rc;
  return status;
}

// Largest eigenvalue of the Gauss-Newton matrix Re(J~^H W^T W J~) (Sec. 3, eq.
// normal_system_discrete2 without eps I, scaled control) by power iteration
// from the constant vector: v_0 = 1/||1||; w = G v_{k-1}; lambda_k = v_{k-1} . w;
// v_k = w / ||w||.  Returns lambda_iters.  With several instances this is the
// block-diagonal matrix of all of them (the largest over instances).
int Ctx::normal_lambda_max(const fwi_opts &o, int iters, double *lambda, fwi_stats *stats) {
  if (!have_fwd) fail(FWI_E_INVAL, "fwi_normal_lambda_max needs fwi_forward at the current model");
  if (iters < 1) fail(FWI_E_INVAL, "iters must be >= 1");
  const long long nc = Nc;
  NormalOp N(*this, o, stats);
  DBuf<double> v, w;
  v.alloc(nc); w.alloc(nc);
  std::vector<double> one((size_t)nc, 1.0 / std::sqrt((double)nc));
  CK(cudaMemcpyAsync(v.p, one.data(), nc * sizeof(double), cudaMemcpyHostToDevice, st));
  double lam = 0.0;
  for (int k = 0; k < iters; ++k) {
    N.apply(v.p, 0.0, w.p);
    lam = N.dot(v.p, w.p);
    const double wn = std::sqrt(N.dot(w.p, w.p));
    if (!std::isfinite(wn)) fail(FWI_E_NUMERIC, "non-finite power iterate");
    if (!(wn > 0.0)) { lam = 0.0; break; }
    KPROF("k_axpby", -1, 24.0 * nc, st);
    k_axpby<double><<<FLAT_BLOCKS, FLAT_THREADS, 0, st>>>(nc, 1.0 / wn, w.p, 0.0, v.p);
    KCHECK();
  }
  sync();
  *lambda = lam;
  return N.solve_rc;
}

// H~ v = eps v + Re(P~^H A'^{-H} F A'^{-1} P~ v) (Sec. 3, eq.
// normal_system_discrete_sum, scaled control): one forward and one adjoint
// refined solve of every block.
int Ctx::hessian_apply(const fwi_opts &o, const double *v, double *hv, int on_device, fwi_stats *stats) {
  if (!have_fwd) fail(FWI_E_INVAL, "fwi_hessian_apply needs fwi_forward at the current model");
  if (!(o.eps >= 0.0)) fail(FWI_E_INVAL, "eps must be >= 0");
  NormalOp N(*this, o, stats);
  DBuf<double> dv, dh;
  const double *vin = v;
  double *out = hv;
  if (!on_device) {
    dv.alloc(Nc); dh.alloc(Nc);
    CK(cudaMemcpyAsync(dv.p, v, Nc * sizeof(double), cudaMemcpyHostToDevice, st));
    vin = dv.p; out = dh.p;
  }
  N.apply(vin, o.eps, out);
  if (!on_device) CK(cudaMemcpyAsync(hv, dh.p, Nc * sizeof(double), cudaMemcpyDeviceToHost, st));
  sync();
  return N.solve_rc;
}

int Ctx::rsgn_step(const fwi_opts &o, double *ds, int on_device, fwi_stats *stats) {
  auto t0 = std::chrono::steady_clock::now();
  build_hierarchy(o);
  if (stats) stats->t_setup_ms += std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  forward(o, stats);
  int rc = rsgn_solve(o, stats);
  apply_update(ds, on_device);
  return rc;
}

}  // namespace fwi

// ==========================================================================
// C ABI
// ==========================================================================
using fwi::Ctx;
using fwi::Err;

struct fwi_ctx {
  Ctx c;
};

static std::string g_create_error;

#define API_BEGIN(ctx)                       \
  if (!(ctx)) return FWI_E_INVAL;            \
  (ctx)->c.err.clear();                      \
  try {
#define API_END(ctx)                         \
  }                                          \
  catch (const Err &e) {                     \
    (ctx)->c.err = e.msg;                    \
    return e.code;                           \
  }                                          \
  catch (const std::exception &e) {          \
    (ctx)->c.err = e.what();                 \
    return FWI_E_INVAL;                      \
  }

static int check_opts(const fwi_opts *o) {
  if (!o) return 0;
  if (o->restart < 1 || o->restart > 200 || o->nu1 < 0 || o->nu2 < 0 || o->mg_cycle < 1 || o->mg_cycle > 2 || o->mg_wdepth < 0 ||
      o->inner_iters < 1 || o->fwd_iters < 1 || !(o->tol > 0.0) || o->max_outer < 1 ||
      (o->precision != FWI_C128 && o->precision != FWI_C64_REFINE) || o->mg_wdepth > MAX_LEVELS ||
      o->arnoldi_dots < FWI_DOT_RUNS || o->arnoldi_dots > FWI_DOT_COMP || o->strip_rows < 2 ||
      o->strip_rows > 64 || (o->coarse_threads != 512 && o->coarse_threads != 1024) || o->outer_solver < 0 ||
      o->outer_solver > 1 || o->inner_solver < 0 || o->inner_solver > 2 || o->hblock < 0 || o->hblock > 1)
    return 0;
  return 1;
}

extern "C" {

void fwi_default_opts(fwi_opts *o) {
  if (!o) return;
  o->precision = FWI_C64_REFINE;
  o->eps = 1e-3;
  o->include_Ls_n = 1;
  o->tol = 1e-6;
  o->restart = 30;
  o->max_outer = 600;
  o->sweep_tol = 1e-3;
  o->max_refine = 8;
  o->inner_iters = 4;
  o->inner_tol = 0.0;
  o->mg_cycle = 2;
  o->mg_wdepth = 2;
  o->nu1 = 2;
  o->nu2 = 2;
  o->omega_jac = 0.5;
  o->shift_beta = 0.5;
  o->sigma_cap = 1.0;
  o->mg_levels = 0;
  o->fwd_tol = 1e-9;
  o->fwd_iters = 60;
  o->max_fwd_refine = 20;
  o->use_graph = 1;
  o->arnoldi_dots = FWI_DOT_COMP;
  o->strip_rows = 16;
  o->fwd_warm = 1;
  o->outer_solver = 0;
  o->inner_solver = 0;
  o->hblock = 0;
  o->coarse_threads = 512;
  o->check_orth = 0;
}

int fwi_create(fwi_ctx **out, int n_instances, const fwi_grid *grids, void *cuda_stream) {
  if (!out) return FWI_E_INVAL;
  *out = nullptr;
  g_create_error.clear();
  if (n_instances < 1 || !grids) { g_create_error = "n_instances >= 1 and grids required"; return FWI_E_INVAL; }
  for (int i = 0; i < n_instances; ++i) {
    const fwi_grid &g = grids[i];
    if (g.nx < 2 || g.nz < 2 || g.npml < 0 || !(g.h > 0.0) ||
        (g.npml > 0 && (!(g.pml_c > 0.0) || !(g.pml_R > 0.0) || !(g.pml_R < 1.0)))) {
      g_create_error = "invalid grid of instance " + std::to_string(i);
      return FWI_E_INVAL;
    }
  }
  fwi_ctx *c = new (std::nothrow) fwi_ctx;
  if (!c) return FWI_E_NOMEM;
  c->c.st = (cudaStream_t)cuda_stream;
  c->c.inst.resize(n_instances);
  for (int i = 0; i < n_instances; ++i) {
    fwi::Instance &I = c->c.inst[i];
    I.g = grids[i];
    I.Nx = grids[i].nx + 2 * grids[i].npml;
    I.Nz = grids[i].nz + 2 * grids[i].npml;
  }
  *out = c;
  return FWI_OK;
}

int fwi_set_survey(fwi_ctx *ctx, int inst, int n_freq, const double *freq_hz, int n_src, const int *src_ix,
                   const int *src_iz, const double *src_amp, const int *rec_offsets, const int *rec_ix,
                   const int *rec_iz, const double *rec_weight) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (inst < 0 || inst >= (int)c.inst.size()) fwi::fail(FWI_E_INVAL, "instance index out of range");
  if (n_freq < 1 || n_src < 1 || !freq_hz || !src_ix || !src_iz || !src_amp || !rec_offsets)
    fwi::fail(FWI_E_INVAL, "bad survey arguments");
  fwi::Instance &I = c.inst[inst];
  for (int f = 0; f < n_freq; ++f)
    if (!(freq_hz[f] > 0.0)) fwi::fail(FWI_E_INVAL, "frequencies must be > 0");
  for (int k = 0; k < n_src; ++k)
    if (src_ix[k] < 0 || src_ix[k] >= I.g.nx || src_iz[k] < 0 || src_iz[k] >= I.g.nz)
      fwi::fail(FWI_E_INVAL, "source outside the core");
  if (rec_offsets[0] != 0) fwi::fail(FWI_E_INVAL, "rec_offsets[0] must be 0");
  for (int k = 0; k < n_src; ++k)
    if (rec_offsets[k + 1] < rec_offsets[k]) fwi::fail(FWI_E_INVAL, "rec_offsets must be non-decreasing");
  int nr = rec_offsets[n_src];
  if (nr > 0 && (!rec_ix || !rec_iz)) fwi::fail(FWI_E_INVAL, "receiver arrays missing");
  for (int e = 0; e < nr; ++e)
    if (rec_ix[e] < 0 || rec_ix[e] >= I.g.nx || rec_iz[e] < 0 || rec_iz[e] >= I.g.nz)
      fwi::fail(FWI_E_INVAL, "receiver outside the core");
  I.freqs.assign(freq_hz, freq_hz + n_freq);
  I.n_src = n_src;
  I.src_ix.assign(src_ix, src_ix + n_src);
  I.src_iz.assign(src_iz, src_iz + n_src);
  I.src_amp.assign(src_amp, src_amp + 2 * n_src);
  I.rec_off.assign(rec_offsets, rec_offsets + n_src + 1);
  I.rec_ix.assign(rec_ix, rec_ix + nr);
  I.rec_iz.assign(rec_iz, rec_iz + nr);
  I.rec_w.assign(nr, 1.0);
  if (rec_weight) I.rec_w.assign(rec_weight, rec_weight + nr);
  I.has_survey = true;
  I.has_data = false;
  c.layout_ok = false;
  c.have_fwd = false;
  return FWI_OK;
  API_END(ctx)
}

int fwi_set_model(fwi_ctx *ctx, int inst, const double *gamma_core, double gamma_ref, int on_device) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (inst < 0 || inst >= (int)c.inst.size() || !gamma_core) fwi::fail(FWI_E_INVAL, "bad model arguments");
  fwi::Instance &I = c.inst[inst];
  size_t n = (size_t)I.g.nx * I.g.nz;
  double sum = 0.0;
  if (on_device) {
    // validate on the device; only the sum and a flag come back
    I.s.alloc(n);
    CK(cudaMemcpyAsync(I.s.p, gamma_core, n * sizeof(double), cudaMemcpyDeviceToDevice, c.st));
    fwi::DBuf<double> part;
    part.alloc(FLAT_BLOCKS + 1);
    fwi::DBuf<int> flag;
    flag.alloc(1);
    flag.zero(c.st);
    KPROF("k_model_stats", -1, 8.0 * n, c.st);
    fwi::k_model_stats<<<FLAT_BLOCKS, FLAT_THREADS, 0, c.st>>>((long long)n, I.s.p, part.p, flag.p);
    KCHECK();
    KPROF("k_reduce_partials", -1, 0, c.st);
    fwi::k_reduce_partials<<<1, 32, 0, c.st>>>(1, FLAT_BLOCKS, part.p, part.p + FLAT_BLOCKS, 0);
    KCHECK();
    int hf = 0;
    CK(cudaMemcpyAsync(&sum, part.p + FLAT_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost, c.st));
    CK(cudaMemcpyAsync(&hf, flag.p, sizeof(int), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    if (hf || !std::isfinite(sum)) fwi::fail(FWI_E_NUMERIC, "gamma must be finite and > 0");
  } else {
    std::vector<double> h(gamma_core, gamma_core + n);
    for (double v : h) {
      if (!std::isfinite(v) || !(v > 0.0)) fwi::fail(FWI_E_NUMERIC, "gamma must be finite and > 0");
      sum += v;
    }
    I.s.upload(h, c.st);
  }
  if (!I.has_model) {
    I.gamma_ref = gamma_ref > 0.0 ? gamma_ref : sum / (double)n;
    I.layer.alloc((size_t)I.Nx * I.Nz);
    KPROF("k_gamma_pad", -1, 0, c.st);
    fwi::k_gamma_pad<<<fwi::grid_for((long long)I.Nx * I.Nz, 256), 256, 0, c.st>>>(I.s.p, I.Nx, I.Nz, I.g.npml,
                                                                                   I.g.nx, I.g.nz, I.layer.p);
    KCHECK();
  } else if (gamma_ref > 0.0) {
    I.gamma_ref = gamma_ref;
  }
  c.sync();
  bool first = !I.has_model;
  I.has_model = true;
  ++c.model_version;
  c.have_fwd = false;
  if (first) c.layout_ok = false;
  return FWI_OK;
  API_END(ctx)
}

int fwi_get_model(fwi_ctx *ctx, int inst, double *gamma_core) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (inst < 0 || inst >= (int)c.inst.size() || !gamma_core || !c.inst[inst].has_model)
    fwi::fail(FWI_E_INVAL, "bad arguments or no model");
  fwi::Instance &I = c.inst[inst];
  CK(cudaMemcpyAsync(gamma_core, I.s.p, (size_t)I.g.nx * I.g.nz * sizeof(double), cudaMemcpyDeviceToHost, c.st));
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

int fwi_set_observed(fwi_ctx *ctx, int inst, const double *d, int on_device) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (inst < 0 || inst >= (int)c.inst.size() || !d) fwi::fail(FWI_E_INVAL, "bad data arguments");
  fwi::Instance &I = c.inst[inst];
  if (!I.has_survey) fwi::fail(FWI_E_INVAL, "set the survey first");
  size_t n = I.freqs.size() * (size_t)I.rec_total();
  I.d.alloc(std::max<size_t>(n, 1));
  if (n) CK(cudaMemcpyAsync(I.d.p, d, n * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.st));
  c.sync();
  I.has_data = true;
  return FWI_OK;
  API_END(ctx)
}

int fwi_forward(fwi_ctx *ctx, const fwi_opts *opts, double *d_pred, double *misfit, fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid options");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  c.forward(o, stats);
  if (d_pred) {
    // entries are in block order; write [inst][f][rec_total]
    std::vector<double2> hq(std::max<size_t>(1, c.rec_node.size()));
    if (!c.rec_node.empty())
      CK(cudaMemcpyAsync(hq.data(), c.q.p, c.rec_node.size() * sizeof(double2), cudaMemcpyDeviceToHost, c.st));
    c.sync();
    size_t e = 0, base = 0;
    for (size_t i = 0; i < c.inst.size(); ++i) {
      fwi::Instance &I = c.inst[i];
      for (size_t f = 0; f < I.freqs.size(); ++f)
        for (int k = 0; k < I.n_src; ++k)
          for (int q = I.rec_off[k]; q < I.rec_off[k + 1]; ++q, ++e) {
            size_t o2 = base + f * I.rec_total() + q;
            d_pred[2 * o2] = hq[e].x;
            d_pred[2 * o2 + 1] = hq[e].y;
          }
      base += I.freqs.size() * I.rec_total();
    }
  }
  if (misfit)
    for (size_t i = 0; i < c.inst.size(); ++i) misfit[i] = c.misfit[i];
  return FWI_OK;
  API_END(ctx)
}

int fwi_get_wavefields(fwi_ctx *ctx, double *u_device) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (!c.have_fwd || !u_device) fwi::fail(FWI_E_INVAL, "no forward wavefields");
  CK(cudaMemcpyAsync(u_device, c.u64.p, c.F0 * sizeof(double2), cudaMemcpyDeviceToDevice, c.st));
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

int fwi_gradient(fwi_ctx *ctx, const fwi_opts *opts, double *misfit, double *grad, int on_device, fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o) || !grad) fwi::fail(FWI_E_INVAL, "invalid arguments");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  return c.gradient(o, misfit, grad, on_device, stats);
  API_END(ctx)
}

int fwi_kkt_solve(fwi_ctx *ctx, const fwi_opts *opts, double *ds, int on_device, fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid options");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  c.build_hierarchy(o);
  int rc = c.kkt_solve(o, stats);
  if (ds) {
    std::vector<double> gr;
    for (auto &I : c.inst) gr.push_back(I.gamma_ref);
    c.write_ctrl(c.xi64.p + 4 * c.F0, ds, on_device, gr.data());
  }
  if (rc != FWI_OK) c.err = "KKT solve stopped at the iteration cap";
  return rc;
  API_END(ctx)
}

int fwi_newton_step(fwi_ctx *ctx, const fwi_opts *opts, double *ds, int on_device, fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid options");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  int rc = c.newton_step(o, ds, on_device, stats);
  if (rc != FWI_OK) c.err = "KKT solve stopped at the iteration cap";
  return rc;
  API_END(ctx)
}

int fwi_rsgn_step(fwi_ctx *ctx, const fwi_opts *opts, double *ds, int on_device, fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid options");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  int rc = c.rsgn_step(o, ds, on_device, stats);
  if (rc == FWI_E_NOCONV) c.err = "reduced-space CG stopped at the iteration cap (or a block solve missed fwd_tol)";
  return rc;
  API_END(ctx)
}

int fwi_normal_lambda_max(fwi_ctx *ctx, const fwi_opts *opts, int iters, double *lambda, fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o) || !lambda) fwi::fail(FWI_E_INVAL, "invalid arguments");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  c.build_hierarchy(o);
  int rc = c.normal_lambda_max(o, iters, lambda, stats);
  if (rc != FWI_OK) c.err = "a block solve of the power iteration missed fwd_tol";
  return rc;
  API_END(ctx)
}

int fwi_hessian_apply(fwi_ctx *ctx, const fwi_opts *opts, const double *v, double *hv, int on_device,
                      fwi_stats *stats) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!check_opts(&o) || !v || !hv) fwi::fail(FWI_E_INVAL, "invalid arguments");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  c.build_hierarchy(o);
  int rc = c.hessian_apply(o, v, hv, on_device, stats);
  if (rc != FWI_OK) c.err = "a block solve of the Hessian product missed fwd_tol";
  return rc;
  API_END(ctx)
}

int fwi_hblock_set(fwi_ctx *ctx, int m, const double *S, const double *Y, int on_device) {
  API_BEGIN(ctx)
  ctx->c.hblock_set(m, S, Y, on_device);
  return FWI_OK;
  API_END(ctx)
}

int fwi_apply_helmholtz(fwi_ctx *ctx, const void *x, void *y, int adjoint, int precision) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (!x || !y) fwi::fail(FWI_E_INVAL, "null buffer");
  fwi_opts o;
  fwi_default_opts(&o);
  c.build_hierarchy(o);
  if (precision == FWI_C128)
    c.field_op<double>(fwi::FM_APPLY, adjoint ? 1 : 0, 0.0, (const double2 *)x, nullptr, (double2 *)y, true, 0);
  else if (precision == FWI_C64_REFINE)
    c.field_op<float>(fwi::FM_APPLY, adjoint ? 1 : 0, 0.0f, (const float2 *)x, nullptr, (float2 *)y, true, 0);
  else fwi::fail(FWI_E_INVAL, "bad precision");
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

int fwi_apply_kkt(fwi_ctx *ctx, const fwi_opts *opts, const void *xi, void *y, int precision) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!xi || !y) fwi::fail(FWI_E_INVAL, "null buffer");
  if (!c.have_fwd) fwi::fail(FWI_E_INVAL, "fwi_apply_kkt needs fwi_forward");
  c.build_hierarchy(o);
  if (precision == FWI_C128) c.kkt_matvec<double>((const double *)xi, (double *)y, o.eps, c.u_T<double>());
  else if (precision == FWI_C64_REFINE) {
    c.ensure_work<float>(o);
    c.kkt_matvec<float>((const float *)xi, (float *)y, o.eps, c.u_T<float>());
  } else fwi::fail(FWI_E_INVAL, "bad precision");
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

int fwi_apply_precond(fwi_ctx *ctx, const fwi_opts *opts, const void *v, void *z, int precision) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!v || !z || !check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid arguments");
  if (!c.have_fwd) fwi::fail(FWI_E_INVAL, "fwi_apply_precond needs fwi_forward");
  c.build_hierarchy(o);
  if (o.inner_solver >= 1) c.ensure_ilu();
  c.hblock_prepare(o);
  long long cnt = 0;
  if (precision == FWI_C128) {
    c.ensure_work<double>(o);
    c.precond<double>((const double *)v, (double *)z, o, &cnt, c.u_T<double>());
  } else if (precision == FWI_C64_REFINE) {
    c.ensure_work<float>(o);
    c.precond<float>((const float *)v, (float *)z, o, &cnt, c.u_T<float>());
  } else fwi::fail(FWI_E_INVAL, "bad precision");
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

int fwi_inner_solve(fwi_ctx *ctx, const fwi_opts *opts, const void *b, void *x, int adjoint, int precision) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!b || !x || !check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid arguments");
  c.build_hierarchy(o);
  if (o.inner_solver >= 1) c.ensure_ilu();
  int iters = o.inner_iters;
  long long cnt = 0;
  if (precision == FWI_C128) {
    c.ensure_work<double>(o);
    c.inner_solve<double>((const double2 *)b, (double2 *)x, adjoint ? 1 : 0, iters, o.inner_tol, o, &cnt,
                          o.inner_solver >= 1);
  } else if (precision == FWI_C64_REFINE) {
    c.ensure_work<float>(o);
    c.inner_solve<float>((const float2 *)b, (float2 *)x, adjoint ? 1 : 0, iters, o.inner_tol, o, &cnt,
                         o.inner_solver >= 1);
  } else fwi::fail(FWI_E_INVAL, "bad precision");
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

int fwi_mg_cycle(fwi_ctx *ctx, const fwi_opts *opts, const void *b, void *x, int precision) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!b || !x || !check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid arguments");
  c.build_hierarchy(o);
  if (precision == FWI_C128) {
    c.ensure_work<double>(o);
    c.mg_cycle<double>((const double2 *)b, (double2 *)x, 0, o);
  } else if (precision == FWI_C64_REFINE) {
    c.ensure_work<float>(o);
    c.mg_cycle<float>((const float2 *)b, (float2 *)x, 0, o);
  } else fwi::fail(FWI_E_INVAL, "bad precision");
  c.sync();
  return FWI_OK;
  API_END(ctx)
}

// ---- multigrid cycle without device allocation ---------------------------
// Scratch of fwi_mg_cycle_noalloc: the level buffers of one multigrid cycle.
// Device code could name it directly; host code only ever holds its device
// address, obtained per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[FWI_NOALLOC_SCRATCH_BYTES];
static void *g_noalloc_addr[256];
static bool g_noalloc_ready[256];

}  // extern "C"

template <typename T>
static int mg_cycle_noalloc_impl(fwi::Ctx &c, const fwi_opts &o, const void *b, void *x) {
  typedef typename fwi::cplx<T>::t T2;
  // buffers: level-0 ping-pong buffer + x, b, t of every global coarse level,
  // each rounded up to 256 bytes
  auto up = [](size_t n) { return (n + 255) / 256 * 256; };
  size_t need = up(c.F0 * sizeof(T2));
  const int lsT = c.ls_p[sizeof(T) == 8];
  for (int l = 1; l <= lsT && l < c.nlev_max; ++l) need += 3 * up(c.lv[l].field * sizeof(T2));
  if (need > (size_t)FWI_NOALLOC_SCRATCH_BYTES)
    fwi::fail(FWI_E_INVAL, "fwi_mg_cycle_noalloc: the batch needs " + std::to_string(need) +
                               " bytes of scratch, more than FWI_NOALLOC_SCRATCH_BYTES (" +
                               std::to_string((size_t)FWI_NOALLOC_SCRATCH_BYTES) + ")");
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 256) fwi::fail(FWI_E_INVAL, "device index out of range");
  if (dev != c.dev)
    fwi::fail(FWI_E_INVAL, "fwi_mg_cycle_noalloc: the context's device (" + std::to_string(c.dev) +
                               ") is not the current device (" + std::to_string(dev) + ")");
  if (!g_noalloc_ready[dev]) {
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      fwi::fail(FWI_E_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_addr[dev] = ptr;
    g_noalloc_ready[dev] = true;
  }
  unsigned char *base = (unsigned char *)g_noalloc_addr[dev];
  size_t off = 0;
  T2 *t0 = (T2 *)(base + off);
  off += up(c.F0 * sizeof(T2));
  T2 *lx[MAX_LEVELS] = {}, *lb[MAX_LEVELS] = {}, *lt[MAX_LEVELS] = {};
  for (int l = 1; l <= lsT && l < c.nlev_max; ++l) {
    size_t bytes = up(c.lv[l].field * sizeof(T2));
    lx[l] = (T2 *)(base + off); off += bytes;
    lb[l] = (T2 *)(base + off); off += bytes;
    lt[l] = (T2 *)(base + off); off += bytes;
  }
  size_t smem = c.smem_bytes[sizeof(T) == 8];
  if (smem > 48 * 1024) fwi::set_coarse_smem<T>((int)smem);
  // no live stencil timing inside this call: its event buffers are allocated
  // on first use, and this call allocates nothing
  struct TimerBlock {
    fwi::Ctx &c;
    bool prev;
    explicit TimerBlock(fwi::Ctx &cc) : c(cc), prev(cc.timer_blocked) { c.timer_blocked = true; }
    ~TimerBlock() { c.timer_blocked = prev; }
  } block(c);
  c.mg_cycle_into<T>((const T2 *)b, (T2 *)x, 0, o, lx, lb, lt, t0);
  c.sync();
  return FWI_OK;
}

extern "C" {

int fwi_mg_cycle_noalloc(fwi_ctx *ctx, const fwi_opts *opts, const void *b, void *x, int precision) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  fwi_opts o;
  fwi_default_opts(&o);
  if (opts) o = *opts;
  if (!b || !x || !check_opts(&o)) fwi::fail(FWI_E_INVAL, "invalid arguments");
  if (!c.layout_ok || c.hier_key != fwi::hierarchy_key(c.model_version, o))
    fwi::fail(FWI_E_INVAL, "fwi_mg_cycle_noalloc: no multigrid hierarchy for these options and the current "
                           "models; call fwi_mg_cycle (or fwi_forward) with the same options first");
  if (precision == FWI_C128) return mg_cycle_noalloc_impl<double>(c, o, b, x);
  if (precision == FWI_C64_REFINE) return mg_cycle_noalloc_impl<float>(c, o, b, x);
  fwi::fail(FWI_E_INVAL, "bad precision");
  return FWI_E_INVAL;
  API_END(ctx)
}

int fwi_get_layout(fwi_ctx *ctx, fwi_layout_info *info) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (!info) fwi::fail(FWI_E_INVAL, "null info");
  c.build_layout();
  info->n_instances = (int)c.inst.size();
  info->n_blocks = c.B;
  info->field_elems = c.F0;
  info->ctrl_elems = c.Nc;
  info->kkt_elems = c.nkkt;
  return FWI_OK;
  API_END(ctx)
}

unsigned long long fwi_kernel_launches(void) { return fwi::g_launches.load(); }

unsigned long long fwi_memory_calls(void) { return fwi::g_memcalls.load(); }

int fwi_stencil_timer(fwi_ctx *ctx, int enable, double *ms, double *bytes, long long *launches,
                      double *pass_bytes) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (c.st) c.sync();
  if (ms) *ms = c.timer_ms;
  if (bytes) *bytes = c.timer_bytes;
  if (launches) *launches = c.timer_n;
  if (pass_bytes) *pass_bytes = c.timer_pbytes;
  if (enable >= 0) {
    c.timer_on = enable > 0;
    c.timer_ms = 0.0; c.timer_bytes = 0.0; c.timer_pbytes = 0.0; c.timer_n = 0;
  }
  return FWI_OK;
  API_END(ctx)
}

int fwi_kernel_profile(fwi_ctx *ctx, int enable, char *buf, long long buflen) {
  API_BEGIN(ctx)
  Ctx &c = ctx->c;
  if (c.st) c.sync();
  fwi::Prof &P = fwi::g_prof;
  if (P.used) P.harvest();
  if (buf) {
    std::string js = "{\"gap_ms\": " + std::to_string(P.gap_ms) + ", \"gaps\": " + std::to_string(P.gaps) +
                     ", \"rows\": [";
    bool first = true;
    char line[512];
    for (auto &kv : P.rows) {
      snprintf(line, sizeof line, "%s{\"kernel\": \"%s\", \"level\": %d, \"launches\": %lld, \"ms\": %.6f, \"bytes\": %.1f}",
               first ? "" : ", ", kv.first.first.c_str(), kv.first.second, kv.second.n, kv.second.ms, kv.second.bytes);
      js += line;
      first = false;
    }
    js += "]}";
    if ((long long)js.size() + 1 > buflen)
      fwi::fail(FWI_E_INVAL, "fwi_kernel_profile: buffer too small, need " + std::to_string(js.size() + 1) + " bytes");
    std::memcpy(buf, js.c_str(), js.size() + 1);
  }
  if (enable >= 0) {
    P.clear();
    P.on = enable > 0;
  }
  return FWI_OK;
  API_END(ctx)
}

const char *fwi_last_error(const fwi_ctx *ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->c.err.c_str();
}

void fwi_destroy(fwi_ctx *ctx) {
  if (!ctx) return;
  bool touched = ctx->c.pin != nullptr;
  for (auto &I : ctx->c.inst) touched = touched || I.has_model;
  if (touched) cudaStreamSynchronize(ctx->c.st);
  delete ctx;
}

}  // extern "C"
