// sipo_abi.cu -- solver contexts and the extern "C" entry points of include/sipo.h.
//
// A context owns every device array of one LP instance.  Setup (sipo_create)
// runs entirely on the device: target statistics, region labels, active-ray
// mask, normalised target and Pock-Chambolle preconditioners.  A solve runs
// the restarted Halpern PDHG as one captured CUDA graph per check period
// (one check step followed by check_every - 1 fused steps); the host only
// reads a done flag between graph launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <string>
#include <type_traits>
#include <vector>

#include "sipo.h"
#include "sipo_kernels.cuh"
#include "sipo_launch.h"
#include "sipo_ops.cuh"
#include "sipo_psf.cuh"
#include "sipo_response.cuh"
#include "sipo_schedule.h"

namespace sipo {
namespace {

thread_local std::string g_err;
std::atomic<long long> g_launches{0};

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] void fail(int code, const std::string& msg) { throw Error{code, msg}; }

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    if (e == cudaErrorMemoryAllocation) fail(SIPO_ERR_OOM, std::string(what) + ": out of device memory");
    fail(SIPO_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

int grid_for(long long n) {
  long long g = (n + kThreads - 1) / kThreads;
  return int(std::max<long long>(1, std::min<long long>(g, (long long)device_sms() * 16)));
}

struct SolverBase {
  virtual ~SolverBase() {}
  // fL_dev, fU_dev (Case 1 with explicit bounds, else null): per-voxel dose bounds
  virtual void setup(const float* fT_dev, const float* fL_dev, const float* fU_dev) = 0;
  virtual void begin_solve() = 0;
  virtual void launch_block(long long n) = 0;
  virtual void request_done() = 0;
  // ends the current solve at its last check (status ITER_LIMIT), so that the
  // returned point and the exported state are that check's T(z)
  virtual void stop_at_last_check() = 0;
  virtual bool done_flag() = 0;
  virtual void finish_solve(void* y_out, int loc, sipo_result* res) = 0;
  virtual void project(const void* vol, void* sino, cudaStream_t s) = 0;
  virtual void backproject(const void* sino, void* vol, cudaStream_t s) = 0;
  virtual void psf_apply(const void* in, void* out, int deriv, cudaStream_t s) = 0;
  virtual void psf_grad(const void* sino, const void* vol, double* grad, cudaStream_t s) = 0;
  virtual void set_sigma(const double* sig) = 0;
  virtual void get_array(int which, void* out, int loc) = 0;
  virtual void profile(int iters, double* ms, int n) = 0;
  virtual int compute_dtype() const = 0;
  virtual cudaStream_t strm() const = 0;
  virtual long long period() const = 0;
  virtual long long max_iter() const = 0;
  virtual void set_tolerances(const sipo_tolerances* t) = 0;
  virtual int get_trace(double* out, int max_entries) = 0;
  // batched solves: zero start without a graph, one check period enqueued on
  // `s` (check step + period - 1 fused steps) followed by a copy of the state
  // to the pinned host mirror, and that mirror.  enqueue_period returns the
  // kernels it enqueued without counting them (it is captured into a graph);
  // add_launches counts one launch of that graph.
  virtual void init_for_batch() = 0;
  virtual long long enqueue_period(cudaStream_t s) = 0;
  virtual void add_launches(long long n) = 0;
  virtual const Scal& host_state() const = 0;
  // warm start: the last check's T(z) of a finished solve (device arrays and
  // their element types), a problem fingerprint, and the import of such a point
  struct Point {
    const void *yp, *gp, *lpu, *lpl, *dp;
    int s_dtype, c_dtype;
    Scal st;
  };
  virtual Point point() const = 0;
  virtual int dev() const = 0;
  virtual std::vector<double> fingerprint() const = 0;
  virtual void warm_from(const SolverBase& src) = 0;
  // start from a caller's point (y, lam_up, lam_lo, u~, v~, omega); null duals: zero
  virtual void state_from(const void* y, const void* lam_up, const void* lam_lo, int loc, double u, double v,
                          double omega) = 0;
  // start from src's last returned primal point times `scale` (same geometry)
  virtual void primal_from(const SolverBase& src, double scale, double u, double v) = 0;
  // tests src's last returned dual point as a Farkas ray of this LP (bound-based
  // test); returns 1 if it proves infeasibility, with the slice in *slice
  virtual int farkas_from(const SolverBase& src, int* slice) = 0;
  // throws INVALID_ARG where src's duals cannot be tested against this LP
  virtual void farkas_compatible(const SolverBase& src) const = 0;
  virtual std::vector<double> label_counts() const = 0;
  virtual std::vector<double> geometry_fingerprint() const = 0;
  // the point T(z) of the last check: y, lam_up, lam_lo (compute type) and u~, v~, omega, k
  virtual void state_to(void* y, void* lam_up, void* lam_lo, int loc, double* scalars) = 0;
  // response-domain post-scaling and metrics of the last solve's dose
  virtual void response_metrics(const Richards& M, const float* mT, double alpha, sipo_response_result* out) = 0;
};

// Element conversion of n values of dtype `in_dtype` at `in` into `out`.
template <typename TO>
void convert_from(const void* in, int in_dtype, TO* out, long long n, cudaStream_t s) {
  const int grid = grid_for(n);
  if (in_dtype == SIPO_F64)
    k_convert<double, TO><<<grid, kThreads, 0, s>>>(static_cast<const double*>(in), out, n);
  else if (in_dtype == SIPO_BF16)
    k_convert<__nv_bfloat16, TO><<<grid, kThreads, 0, s>>>(static_cast<const __nv_bfloat16*>(in), out, n);
  else
    k_convert<float, TO><<<grid, kThreads, 0, s>>>(static_cast<const float*>(in), out, n);
}

// Autotuned backprojector tile per problem shape (process-wide cache).
struct TileKey {
  int nx, ny, nz, na, nd, storage, psf;
  bool operator<(const TileKey& o) const {
    return std::tie(nx, ny, nz, na, nd, storage, psf) < std::tie(o.nx, o.ny, o.nz, o.na, o.nd, o.storage, o.psf);
  }
};
std::mutex g_tile_mutex;
std::map<TileKey, int> g_tile_cache;

constexpr int kNumPhases = 7;
const char* kPhaseNames[kNumPhases] = {"scalar_step", "psf_q",       "project_primal", "backproject",
                                       "psf_d",       "dual_update", "check_step"};

template <typename S>
struct Solver final : SolverBase {
  using C = typename Compute<S>::type;

  // configuration
  int nx, ny, nz, na, nd;
  size_t V, SN;
  double vial_r, mu, sigma[3], trunc;
  int R[3];
  std::vector<double> angles;
  sipo_case_params cp;
  sipo_tolerances tol;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int zl = 1;  // z values per lane of the operator kernels (z_lanes)
  int ze = 1;  // z values per thread of the element-wise kernels (G or 1)
  int P = 64;
  bool psf = false;
  int bp_nv = 0;     // backprojector tile table entry

  // device memory
  std::vector<void*> allocs;
  C *cs = nullptr, *ex = nullptr, *ey = nullptr, *es = nullptr;
  int2 *xspan = nullptr, *yspan = nullptr;
  long long r2i = -1;
  C* taps[3] = {nullptr, nullptr, nullptr};
  C* dtaps[3] = {nullptr, nullptr, nullptr};
  float* fT = nullptr;
  uint8_t *lab = nullptr, *mask = nullptr, *act_col = nullptr, *need = nullptr;
  int2* rspan = nullptr;  // per-ray walked span meeting columns in `need`
  NeedBits nbits{};      // `need` packed as bits for the projector
  C *ft = nullptr, *row = nullptr, *col = nullptr;
  C* fu = nullptr;            // Case 1 with explicit bounds: f_U / f_crit on gel
  double fu_sum = 0.0;        // sum_gel f~_U (fingerprint of explicit bounds)
  S *y = nullptr, *y0 = nullptr, *yp = nullptr, *ybar = nullptr;
  C *gp = nullptr, *g0 = nullptr, *gc = nullptr;
  S *lu = nullptr, *ll = nullptr, *lu0 = nullptr, *ll0 = nullptr, *lpu = nullptr, *lpl = nullptr;
  S *q = nullptr, *qp = nullptr, *kq = nullptr;
  C *d = nullptr, *d0 = nullptr, *dp = nullptr;
  C *braw = nullptr, *t1 = nullptr, *t2 = nullptr, *t3 = nullptr, *tvol = nullptr;
  C *cert_b = nullptr, *cert_q = nullptr;  // bound-based certificate: A 1_rows, candidate
  bool cert_on = false;
  double cert_B = 0.0;
  // the certificate slice by slice (no PSF extent along z): B_z, the block
  // partials of obj_z and the per-slice maxima kappa_z
  bool cert_slices = false;
  double *cert_Bz = nullptr, *cert_pz = nullptr;
  unsigned long long* cert_kz = nullptr;
  Scal* st = nullptr;
  double* part = nullptr;
  double* trace = nullptr;
  static constexpr int kTraceCap = 4096;
  Scal* h_st = nullptr;  // pinned host mirror

  // host constants
  bool ft_is_const = false;
  C ft_const = C(0);
  double up_ratio = 0.0, f_crit = 0.0, col_u = 0.0, col_v = 0.0, h_norm = 0.0, c_norm = 0.0;
  double omega0 = 1.0, c_u = 0.0, c_v = 0.0, band_rhs = 0.0;
  long long n_band = 0, n_gel = 0;
  int has_u = 0, has_v = 0;

  cudaGraphExec_t gexec = nullptr;
  long long graph_nodes = 0;
  long long launches = 0;
  bool solved = false;
  std::chrono::steady_clock::time_point t_start;

  template <typename T>
  T* dalloc(size_t n) {
    void* p = nullptr;
    ck(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cudaMalloc");
    allocs.push_back(p);
    return static_cast<T*>(p);
  }

  int device = 0;  // the device current at creation; every array lives there

  Solver(const sipo_geometry* g, const sipo_case_params* c, const sipo_tolerances* t, cudaStream_t s) {
    ck(cudaGetDevice(&device), "cudaGetDevice");
    nx = g->nx; ny = g->ny; nz = g->nz; na = g->n_angles; nd = g->n_det;
    V = size_t(nx) * ny * nz;
    SN = size_t(na) * nd * nz;
    vial_r = g->vial_radius;
    mu = g->mu;
    trunc = g->psf_trunc > 0 ? g->psf_trunc : 4.0;
    for (int a = 0; a < 3; ++a) {
      sigma[a] = g->psf_sigma[a];
      R[a] = sigma[a] > 0 ? int(std::ceil(trunc * sigma[a])) : 0;
    }
    psf = R[0] > 0 || R[1] > 0 || R[2] > 0;
    angles.assign(g->angles, g->angles + na);
    cp = *c;
    tol = *t;
    P = tol.check_every > 0 ? tol.check_every : 64;
    zl = z_lanes<C>(nz);
    ze = zl > 1 ? z_group<C>() : 1;
    if (s) {
      stream = s;
    } else {
      ck(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking), "cudaStreamCreate");
      own_stream = true;
    }
    ck(cudaHostAlloc(reinterpret_cast<void**>(&h_st), sizeof(Scal), cudaHostAllocDefault), "cudaHostAlloc");
  }

  ~Solver() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (stream) cudaStreamSynchronize(stream);
    for (void* p : allocs) cudaFree(p);
    if (tconv) cudaFree(tconv);
    if (h_st) cudaFreeHost(h_st);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }

  int compute_dtype() const override { return sizeof(C) == 8 ? SIPO_F64 : SIPO_F32; }
  cudaStream_t strm() const override { return stream; }
  long long period() const override { return P; }
  long long max_iter() const override { return tol.max_iter; }
  int get_trace(double* out, int max_entries) override {
    ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, stream), "read state");
    ck(cudaStreamSynchronize(stream), "trace");
    const int n = std::min(h_st->trace_n, std::max(0, max_entries));
    if (n > 0) {
      ck(cudaMemcpyAsync(out, trace, size_t(n) * kTraceFields * sizeof(double), cudaMemcpyDeviceToHost, stream),
         "trace");
      ck(cudaStreamSynchronize(stream), "trace");
    }
    return n;
  }

  void init_for_batch() override {
    if (!warm_pending) init_state();
    warm_pending = false;
    launches = 0;
    t_start = std::chrono::steady_clock::now();
  }

  long long enqueue_period(cudaStream_t s) override {
    const long long before = launches;
    enqueue_check(s);
    for (int i = 1; i < P; ++i) enqueue_normal(s);
    ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, s), "state copy");
    const long long k = launches - before;
    launches = before;
    g_launches -= k;
    return k;
  }

  void add_launches(long long n) override { count(n); }

  const Scal& host_state() const override { return *h_st; }

  // ------------------------------------------------------------ warm start
  bool warm_pending = false;

  static int dtype_of_s() {
    return sizeof(S) == 8 ? SIPO_F64 : (sizeof(S) == 2 ? SIPO_BF16 : SIPO_F32);
  }

  int dev() const override { return device; }

  Point point() const override {
    Point pt{yp, gp, lpu, lpl, dp, dtype_of_s(), compute_dtype(), *h_st};
    return pt;
  }

  std::vector<double> fingerprint() const override {
    std::vector<double> f = {double(device), double(nx), double(ny), double(nz), double(na), double(nd),
                             double(cp.kase),
                             double(n_band), double(n_gel), f_crit, cp.tol_lo, cp.tol_hi,
                             cp.inhibit_ratio, double(cp.band_width), psf ? 1.0 : 0.0,
                             fu ? 1.0 : 0.0, fu_sum};
    f.insert(f.end(), angles.begin(), angles.end());
    return f;
  }

  // The next solve starts from src's last T(z): it becomes both the iterate and
  // the restart anchor (exactly what a restart does), with src's primal weight.
  void warm_from(const SolverBase& src) override {
    if (src.fingerprint() != fingerprint())
      fail(SIPO_ERR_INVALID_ARG, "warm start: the two contexts do not hold the same problem on one device");
    ck(cudaStreamSynchronize(src.strm()), "warm start: source");
    const Point pt = src.point();
    if (pt.st.k <= 0 && pt.st.done == 0)
      fail(SIPO_ERR_INVALID_ARG, "warm start: the source context has not been solved");
    init_state();
    convert_from<S>(pt.yp, pt.s_dtype, yp, (long long)SN, stream);
    convert_from<C>(pt.gp, pt.c_dtype, gp, (long long)SN, stream);
    convert_from<S>(pt.lpu, pt.s_dtype, lpu, (long long)V, stream);
    convert_from<S>(pt.lpl, pt.s_dtype, lpl, (long long)V, stream);
    convert_from<C>(pt.dp, pt.c_dtype, dp, (long long)V, stream);
    Scal h = *h_st;
    h.u = h.u0 = h.up = pt.st.up;
    h.v = h.v0 = h.vp = pt.st.vp;
    h.omega = pt.st.omega;
    h.restart = 1;
    *h_st = h;
    ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
    // the copy reads the pinned mirror when it runs: finish it before the
    // mirror is written again below
    ck(cudaStreamSynchronize(stream), "warm start");
    const Bufs<S, C> B = bufs();
    const long long nvv = (long long)(V / ze), nvs = (long long)(SN / ze);
    if (ze > 1) {
      k_blend_sino<S, C, z_group<C>()><<<grid_for(nvs), kThreads, 0, stream>>>(B, nvs);
      k_blend_vol<S, C, z_group<C>()><<<kRedBlocks, kThreads, 0, stream>>>(B, nvv);
    } else {
      k_blend_sino<S, C, 1><<<grid_for(nvs), kThreads, 0, stream>>>(B, nvs);
      k_blend_vol<S, C, 1><<<kRedBlocks, kThreads, 0, stream>>>(B, nvv);
    }
    h.restart = 0;
    *h_st = h;
    ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
    ck(cudaStreamSynchronize(stream), "warm start");
    count(7);
    warm_pending = true;
  }

  // The next solve starts from a caller's point: y (compute type,
  // [n_angles][n_det][nz]) projected onto y >= 0 and the active rays; the
  // duals lam_up, lam_lo ([ny][nx][nz], null: zero) projected onto their
  // domain; the scalars u~ and v~ (a negative or non-finite value: the
  // smallest the point allows, max of A^T y over band rows for u~ and max of
  // A^T y / f~ over gel rows, at least 1, for v~); the primal weight omega
  // (<= 0 or non-finite: the default).  The point becomes iterate and restart
  // anchor, as after a restart; A^T y and A (lam_up - lam_lo) are recomputed.
  void state_from(const void* y_in, const void* up_in, const void* lo_in, int loc, double u, double v,
                  double omega) override {
    const cudaMemcpyKind kind = loc == SIPO_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    init_state();
    C* ts = nullptr;
    ck(cudaMallocAsync(reinterpret_cast<void**>(&ts), SN * sizeof(C), stream), "state tmp");
    ck(cudaMemcpyAsync(ts, y_in, SN * sizeof(C), kind, stream), "state y");
    start_from(ts, 1.0, up_in, lo_in, loc, u, v, omega);
  }

  std::vector<double> geometry_fingerprint() const override {
    std::vector<double> f = {double(device), double(nx), double(ny), double(nz), double(na), double(nd),
                             vial_r, mu, sigma[0], sigma[1], sigma[2], trunc};
    f.insert(f.end(), angles.begin(), angles.end());
    return f;
  }

  // The two-stage transfer on the device: src's returned point y (its last
  // T(z), in src's storage type) times `scale` becomes this context's primal
  // start, as sipo_set_primal would make it from a copy of it.
  void primal_from(const SolverBase& src, double scale, double u, double v) override {
    if (src.geometry_fingerprint() != geometry_fingerprint())
      fail(SIPO_ERR_INVALID_ARG, "primal transfer: the contexts differ in geometry or device");
    ck(cudaStreamSynchronize(src.strm()), "primal transfer: source");
    const Point pt = src.point();
    if (pt.st.k <= 0 && pt.st.done == 0)
      fail(SIPO_ERR_INVALID_ARG, "primal transfer: the source context has not been solved");
    init_state();
    C* ts = nullptr;
    ck(cudaMallocAsync(reinterpret_cast<void**>(&ts), SN * sizeof(C), stream), "state tmp");
    convert_from<C>(pt.yp, pt.s_dtype, ts, (long long)SN, stream);
    count(1);
    start_from(ts, scale, nullptr, nullptr, SIPO_DEVICE, u, v, -1.0);
  }

  std::vector<double> label_counts() const override { return {double(n_band), double(n_gel)}; }

  // The dual point T(z) of src's last check (lam_up, lam_lo) becomes the
  // candidate of the bound-based certificate of this context's LP (the epoch
  // difference with a zero anchor) and is tested once, slice by slice where
  // the operator allows.  The candidate's scale does not matter (the test is
  // homogeneous), so src may hold another normalisation of the same part, e.g.
  // the general form with w2 = 0 whose optimum u~* is the best achievable
  // band-to-gel ratio: its optimal dual, tested in Case 2 at a ratio below u~*,
  // is a Farkas ray.  Resets this context's solver state.
  void farkas_compatible(const SolverBase& src) const override {
    if (src.geometry_fingerprint() != geometry_fingerprint() || src.label_counts() != label_counts())
      fail(SIPO_ERR_INVALID_ARG, "Farkas test: the contexts differ in geometry, device or labels");
    if (!cert_on) fail(SIPO_ERR_INVALID_ARG, "Farkas test: the general form has no bound-based certificate");
  }

  int farkas_from(const SolverBase& src, int* slice) override {
    farkas_compatible(src);
    ck(cudaStreamSynchronize(src.strm()), "Farkas test: source");
    const Point pt = src.point();
    if (pt.st.k <= 0 && pt.st.done == 0)
      fail(SIPO_ERR_INVALID_ARG, "Farkas test: the source context has not been solved");
    init_state();  // zero anchors lu0, ll0: the candidate is lam itself
    convert_from<S>(pt.lpu, pt.s_dtype, lpu, (long long)V, stream);
    convert_from<S>(pt.lpl, pt.s_dtype, lpl, (long long)V, stream);
    count(2);
    enqueue_certificate(stream);
    ck(cudaGetLastError(), "Farkas test");
    ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, stream), "read state");
    ck(cudaStreamSynchronize(stream), "Farkas test");
    check_bp_fault();
    const int cert = h_st->cert;
    if (slice) *slice = cert ? h_st->cert_z : -1;
    init_state();
    return cert;
  }

  // Shared tail of the starts: ts (device, compute type, SN values, freed
  // here) scaled and projected onto the primal domain becomes y; the duals
  // as in state_from.
  void start_from(C* ts, double scale, const void* up_in, const void* lo_in, int loc, double u, double v,
                  double omega) {
    const Geo<C> g = geo();
    const Bufs<S, C> B = bufs();
    const cudaMemcpyKind kind = loc == SIPO_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    k_import_primal<S, C><<<grid_for((long long)SN), kThreads, 0, stream>>>(ts, col, yp, C(scale), (long long)SN);
    ck(cudaFreeAsync(ts, stream), "free");
    // d = A^T y with the operator of a check step's plain backprojection
    launch_backproject<S, S, C, kBpStore, C>(g, yp, B, psf ? braw : dp, need, zl, stream, bp_nv);
    if (psf) psf3<C, C>(braw, dp, t1, t2, -1, stream);
    count(2);
    if (up_in || lo_in) {
      C *tu = nullptr, *tl = nullptr, *tq = nullptr;
      ck(cudaMallocAsync(reinterpret_cast<void**>(&tu), V * sizeof(C), stream), "state tmp");
      ck(cudaMallocAsync(reinterpret_cast<void**>(&tl), V * sizeof(C), stream), "state tmp");
      ck(cudaMallocAsync(reinterpret_cast<void**>(&tq), V * sizeof(C), stream), "state tmp");
      if (up_in) ck(cudaMemcpyAsync(tu, up_in, V * sizeof(C), kind, stream), "state lam_up");
      else ck(cudaMemsetAsync(tu, 0, V * sizeof(C), stream), "memset");
      if (lo_in) ck(cudaMemcpyAsync(tl, lo_in, V * sizeof(C), kind, stream), "state lam_lo");
      else ck(cudaMemsetAsync(tl, 0, V * sizeof(C), stream), "memset");
      k_import_dual<S, C><<<grid_for((long long)V), kThreads, 0, stream>>>(tu, tl, lab, lpu, lpl, tq,
                                                                          (long long)V);
      count(1);
      // A q of the imported duals on the active rays (the T point's g)
      project(tq, gp, stream);
      k_apply_mask<C><<<grid_for((long long)SN), kThreads, 0, stream>>>(gp, mask, (long long)SN);
      count(1);
      ck(cudaFreeAsync(tu, stream), "free");
      ck(cudaFreeAsync(tl, stream), "free");
      ck(cudaFreeAsync(tq, stream), "free");
    }
    const bool need_u = has_u && !(u >= 0.0 && std::isfinite(u));
    const bool need_v = has_v && !(v >= 1.0 && std::isfinite(v));
    if (need_u || need_v) {
      k_metrics<C><<<kRedBlocks, kThreads, 0, stream>>>(dp, lab, fT, ft_is_const ? nullptr : ft, ft_const, f_crit,
                                                       (long long)V, part);
      count(1);
      std::vector<double> hp(8 * size_t(kRedBlocks));
      ck(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, stream), "start");
      ck(cudaStreamSynchronize(stream), "state start");
      double mx_band = 0.0, mx_gel = 1.0;
      for (int b = 0; b < kRedBlocks; ++b) {
        mx_band = std::max(mx_band, hp[2 * kRedBlocks + b]);
        mx_gel = std::max(mx_gel, hp[7 * kRedBlocks + b]);
      }
      if (need_u) u = mx_band;
      if (need_v) v = mx_gel;
      zero(part, size_t(kNumSlots) * kRedBlocks);
    }
    Scal h = *h_st;
    if (has_u) h.u = h.u0 = h.up = u;
    if (has_v) h.v = h.v0 = h.vp = v;
    if (omega > 0 && std::isfinite(omega)) h.omega = omega;
    h.restart = 1;
    *h_st = h;
    ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
    ck(cudaStreamSynchronize(stream), "state start");
    const long long nvv = (long long)(V / ze), nvs = (long long)(SN / ze);
    if (ze > 1) {
      k_blend_sino<S, C, z_group<C>()><<<grid_for(nvs), kThreads, 0, stream>>>(B, nvs);
      k_blend_vol<S, C, z_group<C>()><<<kRedBlocks, kThreads, 0, stream>>>(B, nvv);
    } else {
      k_blend_sino<S, C, 1><<<grid_for(nvs), kThreads, 0, stream>>>(B, nvs);
      k_blend_vol<S, C, 1><<<kRedBlocks, kThreads, 0, stream>>>(B, nvv);
    }
    count(2);
    h.restart = 0;
    *h_st = h;
    ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
    ck(cudaStreamSynchronize(stream), "state start");
    warm_pending = true;
  }

  // Checkpoint: the point T(z) of the last check of the most recent solve (the
  // point a warm start or a resume continues from), in the compute type.
  void state_to(void* y_out, void* up_out, void* lo_out, int loc, double* scalars) override {
    ck(cudaStreamSynchronize(stream), "checkpoint");
    if (!solved) fail(SIPO_ERR_INVALID_ARG, "checkpoint: the context has not been solved");
    if (y_out) copy_out(yp, SN, y_out, loc, conv_tmp(SN));
    if (up_out) copy_out(lpu, V, up_out, loc, conv_tmp(V));
    if (lo_out) copy_out(lpl, V, lo_out, loc, conv_tmp(V));
    ck(cudaStreamSynchronize(stream), "checkpoint");
    if (scalars) {
      scalars[0] = h_st->up;
      scalars[1] = h_st->vp;
      scalars[2] = h_st->omega;
      scalars[3] = double(h_st->k);
    }
  }

  // conversion scratch for copies out of BF16 storage (never a state buffer)
  C* tconv = nullptr;
  size_t tconv_n = 0;
  C* conv_tmp(size_t n) {
    if (std::is_same<S, C>::value) return nullptr;
    if (tconv_n < n) {
      if (tconv) {
        ck(cudaStreamSynchronize(stream), "scratch");
        ck(cudaFree(tconv), "scratch");
      }
      ck(cudaMalloc(reinterpret_cast<void**>(&tconv), n * sizeof(C)), "scratch");
      tconv_n = n;
    }
    return tconv;
  }

  // Response-domain back end of the last solve (Sec. 2.7: Eq. 28 with unit
  // weights, Eq. 46): alpha > 0 is used as given; otherwise alpha minimises
  // Phi_m(alpha) = sum_gel (M(alpha d_i) - m_T,i)^2 over a geometric grid of
  // kPhiCand factors spanning 1/16 to 16 times the dose-domain factor of
  // Eq. 27, refined six times on a linear grid between the neighbours of the
  // best candidate (each round shrinks the bracket about 15-fold).
  void response_metrics(const Richards& M, const float* mT_src, double alpha, sipo_response_result* out) override {
    if (!solved) fail(SIPO_ERR_INVALID_ARG, "response metrics need a solved context");
    float* mT = nullptr;
    double *alphas = nullptr, *rp = nullptr;
    const size_t np = size_t(kPhiCand) * kRedBlocks;
    ck(cudaMallocAsync(reinterpret_cast<void**>(&mT), V * sizeof(float), stream), "response tmp");
    ck(cudaMallocAsync(reinterpret_cast<void**>(&alphas), kPhiCand * sizeof(double), stream), "response tmp");
    ck(cudaMallocAsync(reinterpret_cast<void**>(&rp), np * sizeof(double), stream), "response tmp");
    ck(cudaMemcpyAsync(mT, mT_src, V * sizeof(float), cudaMemcpyDefault, stream), "copy m_T");
    std::vector<double> a(kPhiCand), hp(np);
    auto phi_round = [&](int& best, double& best_phi) {
      ck(cudaMemcpyAsync(alphas, a.data(), kPhiCand * sizeof(double), cudaMemcpyHostToDevice, stream), "alphas");
      k_response_phi<C><<<kRedBlocks, kThreads, 0, stream>>>(dp, lab, mT, M, alphas, (long long)V, rp);
      count(1);
      ck(cudaMemcpyAsync(hp.data(), rp, np * sizeof(double), cudaMemcpyDeviceToHost, stream), "phi");
      ck(cudaStreamSynchronize(stream), "phi");
      best = 0;
      best_phi = INFINITY;
      for (int j = 0; j < kPhiCand; ++j) {
        double t = 0.0;
        for (int b = 0; b < kRedBlocks; ++b) t += hp[size_t(j) * kRedBlocks + b];
        if (t < best_phi) { best_phi = t; best = j; }
      }
    };
    double phi = 0.0;
    int best = 0;
    if (alpha > 0) {
      std::fill(a.begin(), a.end(), alpha);
      phi_round(best, phi);
    } else {
      // centre: the dose-domain factor <f~, f_T> / <f~, f~> (Eq. 27)
      k_metrics<C><<<kRedBlocks, kThreads, 0, stream>>>(dp, lab, fT, ft_is_const ? nullptr : ft, ft_const, f_crit,
                                                       (long long)V, part);
      count(1);
      std::vector<double> mp(8 * size_t(kRedBlocks));
      ck(cudaMemcpyAsync(mp.data(), part, mp.size() * sizeof(double), cudaMemcpyDeviceToHost, stream), "metrics");
      ck(cudaStreamSynchronize(stream), "metrics");
      double sdf = 0.0, sdd = 0.0;
      for (int b = 0; b < kRedBlocks; ++b) { sdf += mp[4 * kRedBlocks + b]; sdd += mp[5 * kRedBlocks + b]; }
      const double a0 = (sdf > 0 && sdd > 0) ? sdf / sdd : 1.0;
      for (int j = 0; j < kPhiCand; ++j) a[j] = a0 * std::pow(256.0, double(j) / (kPhiCand - 1)) / 16.0;
      phi_round(best, phi);
      for (int round = 0; round < 6; ++round) {
        const double lo = a[std::max(best - 1, 0)], hi = a[std::min(best + 1, kPhiCand - 1)];
        for (int j = 0; j < kPhiCand; ++j) a[j] = lo + (hi - lo) * double(j) / (kPhiCand - 1);
        phi_round(best, phi);
      }
      alpha = a[best];
    }
    k_response_ratio<C><<<kRedBlocks, kThreads, 0, stream>>>(dp, lab, mT, M, alpha, (long long)V, rp);
    count(1);
    ck(cudaMemcpyAsync(hp.data(), rp, 4 * size_t(kRedBlocks) * sizeof(double), cudaMemcpyDeviceToHost, stream),
       "ratio");
    ck(cudaFreeAsync(mT, stream), "free");
    ck(cudaFreeAsync(alphas, stream), "free");
    ck(cudaFreeAsync(rp, stream), "free");
    ck(cudaStreamSynchronize(stream), "response metrics");
    double v[4] = {1e300, -1e300, -1e300, 1e300};
    for (int b = 0; b < kRedBlocks; ++b) {
      v[0] = std::min(v[0], hp[0 * kRedBlocks + b]);
      v[1] = std::max(v[1], hp[1 * kRedBlocks + b]);
      v[2] = std::max(v[2], hp[2 * kRedBlocks + b]);
      v[3] = std::min(v[3], hp[3 * kRedBlocks + b]);
    }
    std::memset(out, 0, sizeof(*out));
    out->alpha = alpha;
    out->phi = phi;
    out->ratio_min = v[0];
    out->ratio_max = v[1];
    out->dtvr_m = v[0] > 0 ? v[1] / v[0] : INFINITY;
    out->m_band_max = n_band > 0 ? v[2] : 0.0;
    out->m_gel_min = v[3];
    out->psr_m = (n_band > 0 && v[2] > 0) ? v[3] / v[2] : INFINITY;
  }

  void set_tolerances(const sipo_tolerances* t) override {
    const int p = t->check_every > 0 ? t->check_every : 64;
    if (p != P || t->storage != tol.storage)
      fail(SIPO_ERR_INVALID_ARG, "check_every and storage are fixed at creation");
    if (!(t->kkt_tol >= 0) || t->max_iter < 0) fail(SIPO_ERR_INVALID_ARG, "bad tolerances");
    tol.kkt_tol = t->kkt_tol;
    tol.max_iter = t->max_iter;
    if (t->primal_weight > 0) omega0 = t->primal_weight;
    if (warm_pending) {  // the imported state is kept; only the limits change
      h_st->kkt_tol = tol.kkt_tol;
      h_st->max_iter = tol.max_iter;
      ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
      ck(cudaStreamSynchronize(stream), "tolerances");
    }
  }

  Geo<C> geo() const {
    Geo<C> g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.na = na; g.nd = nd;
    g.cx = C((nx - 1) / 2.0);
    g.cy = C((ny - 1) / 2.0);
    g.off = C((nd - 1) / 2.0);
    g.cs = cs; g.ex = ex; g.ey = ey; g.es = es;
    g.vial_r = vial_r;
    g.r2i = r2i;
    g.xspan = xspan;
    g.yspan = yspan;
    return g;
  }

  Bufs<S, C> bufs() const {
    Bufs<S, C> b;
    b.y = y; b.y0 = y0; b.yp = yp; b.ybar = ybar; b.col = col; b.gp = gp; b.g0 = g0; b.gc = gc;
    b.lu = lu; b.ll = ll; b.lu0 = lu0; b.ll0 = ll0; b.lpu = lpu; b.lpl = lpl; b.q = q; b.qp = qp;
    b.d = d; b.d0 = d0; b.dp = dp; b.row = row; b.ft = ft_is_const ? nullptr : ft; b.lab = lab;
    b.ft_const = ft_const; b.up_ratio = C(up_ratio); b.fu = fu; b.has_u = has_u; b.has_v = has_v;
    b.band_rhs = C(band_rhs); b.st = st; b.part = part;
    b.cert_b = cert_b; b.cert_q = cert_q; b.cert_kz = cert_kz;
    return b;
  }

  void count(long long n) {
    launches += n;
    g_launches += n;
  }

  // ------------------------------------------------------------- tables
  void upload_taps() {
    for (int a = 0; a < 3; ++a) {
      if (R[a] == 0) continue;
      std::vector<C> h(2 * R[a] + 1), hd(2 * R[a] + 1);
      std::vector<double> e(2 * R[a] + 1), de(2 * R[a] + 1);
      double S0 = 0, dS = 0;
      for (int i = -R[a]; i <= R[a]; ++i) {
        const double ev = std::exp(-(double(i) * i) / (2.0 * sigma[a] * sigma[a]));
        e[i + R[a]] = ev;
        de[i + R[a]] = ev * double(i) * i / (sigma[a] * sigma[a] * sigma[a]);
        S0 += ev;
        dS += de[i + R[a]];
      }
      for (int i = 0; i < 2 * R[a] + 1; ++i) {
        h[i] = C(e[i] / S0);
        hd[i] = C((de[i] * S0 - e[i] * dS) / (S0 * S0));
      }
      ck(cudaMemcpy(taps[a], h.data(), h.size() * sizeof(C), cudaMemcpyHostToDevice), "taps");
      ck(cudaMemcpy(dtaps[a], hd.data(), hd.size() * sizeof(C), cudaMemcpyHostToDevice), "dtaps");
    }
  }

  // Inside-vial index spans per row and per column, from the exact integer
  // test (2ix - nx + 1)^2 + (2iy - ny + 1)^2 <= floor(4 R^2).
  void build_spans() {
    r2i = vial_r > 0 ? (long long)std::floor(4.0 * (vial_r * vial_r)) : -1;
    std::vector<int2> hx(ny), hy(nx);
    auto inside = [&](int ix, int iy) {
      if (r2i < 0) return true;
      const long long a = 2LL * ix - (nx - 1), b = 2LL * iy - (ny - 1);
      return a * a + b * b <= r2i;
    };
    for (int iy = 0; iy < ny; ++iy) {
      int lo = nx, hi = -1;
      for (int ix = 0; ix < nx; ++ix)
        if (inside(ix, iy)) { lo = std::min(lo, ix); hi = std::max(hi, ix); }
      hx[iy] = make_int2(lo, hi);
    }
    for (int ix = 0; ix < nx; ++ix) {
      int lo = ny, hi = -1;
      for (int iy = 0; iy < ny; ++iy)
        if (inside(ix, iy)) { lo = std::min(lo, iy); hi = std::max(hi, iy); }
      hy[ix] = make_int2(lo, hi);
    }
    xspan = dalloc<int2>(ny);
    yspan = dalloc<int2>(nx);
    ck(cudaMemcpy(xspan, hx.data(), hx.size() * sizeof(int2), cudaMemcpyHostToDevice), "xspan");
    ck(cudaMemcpy(yspan, hy.data(), hy.size() * sizeof(int2), cudaMemcpyHostToDevice), "yspan");
  }

  void build_tables() {
    build_spans();
    std::vector<C> h_cs(2 * size_t(na));
    for (int k = 0; k < na; ++k) {
      h_cs[2 * k] = C(std::cos(angles[k]));
      h_cs[2 * k + 1] = C(std::sin(angles[k]));
    }
    cs = dalloc<C>(h_cs.size());
    ck(cudaMemcpy(cs, h_cs.data(), h_cs.size() * sizeof(C), cudaMemcpyHostToDevice), "cs");
    if (vial_r > 0) {
      const double off = (nd - 1) / 2.0;
      std::vector<C> h_es(size_t(na) * nd);
      for (int k = 0; k < na; ++k)
        for (int j = 0; j < nd; ++j) {
          const double sj = j - off;
          h_es[size_t(k) * nd + j] =
              std::fabs(sj) <= vial_r ? C(std::exp(-mu * std::sqrt(std::max(vial_r * vial_r - sj * sj, 0.0))))
                                      : C(0);
        }
      es = dalloc<C>(h_es.size());
      ck(cudaMemcpy(es, h_es.data(), h_es.size() * sizeof(C), cudaMemcpyHostToDevice), "es");
      if (mu != 0.0) {
        std::vector<C> h_ex(size_t(na) * nx), h_ey(size_t(na) * ny);
        for (int k = 0; k < na; ++k) {
          const double s = std::sin(angles[k]), c = std::cos(angles[k]);
          for (int ix = 0; ix < nx; ++ix) h_ex[size_t(k) * nx + ix] = C(std::exp(mu * (ix - (nx - 1) / 2.0) * s));
          for (int iy = 0; iy < ny; ++iy) h_ey[size_t(k) * ny + iy] = C(std::exp(-mu * (iy - (ny - 1) / 2.0) * c));
        }
        ex = dalloc<C>(h_ex.size());
        ey = dalloc<C>(h_ey.size());
        ck(cudaMemcpy(ex, h_ex.data(), h_ex.size() * sizeof(C), cudaMemcpyHostToDevice), "ex");
        ck(cudaMemcpy(ey, h_ey.data(), h_ey.size() * sizeof(C), cudaMemcpyHostToDevice), "ey");
      }
    }
    for (int a = 0; a < 3; ++a)
      if (R[a] > 0) {
        taps[a] = dalloc<C>(2 * R[a] + 1);
        dtaps[a] = dalloc<C>(2 * R[a] + 1);
      }
    upload_taps();
    if (psf) unit_tap();  // identity axes of a partial PSF, allocated before any capture
  }

  // ---------------------------------------------------------------- PSF
  // in -> out through the three axis passes (taps or, on deriv_axis, their
  // sigma derivative).  tmp_a and tmp_b are C volumes distinct from in/out.
  template <typename TI, typename TO>
  void psf3(const TI* in, TO* out, C* tmp_a, C* tmp_b, int deriv, cudaStream_t s) {
    const C* tp[3];
    for (int a = 0; a < 3; ++a) tp[a] = (deriv == a) ? dtaps[a] : taps[a];
    // an axis without blur runs the single tap 1 (R = 0): a copy
    if constexpr (sizeof(C) == 4) {
      // single precision, nz % 4 == 0: x and y in one pass through shared
      // memory, then z from shared-memory chunks
      const size_t smem = conv_xy_smem(R[0], R[1]);
      if (nz % 4 == 0 && smem <= 227 * 1024 && R[2] <= kZMaxR) {
        const float* tpx = reinterpret_cast<const float*>(tp[0] ? tp[0] : unit_tap());
        const float* tpy = reinterpret_cast<const float*>(tp[1] ? tp[1] : unit_tap());
        const float* tpz = reinterpret_cast<const float*>(tp[2] ? tp[2] : unit_tap());
        const long long tiles = (long long)((ny + kXyT - 1) / kXyT) * ((nx + kXyT - 1) / kXyT) *
                                ((nz / 4 + kXyZG - 1) / kXyZG);
        const long long per_sm = std::max<long long>(1, std::min<long long>(8, (227LL * 1024) / (long long)smem));
        const int gxy = int(std::max<long long>(1, std::min<long long>(tiles, device_sms() * per_sm)));
        launch_conv_xy_fused<TI, C>(in, reinterpret_cast<float*>(tmp_a), tpx, R[0], tpy, R[1], nx, ny, nz, gxy, smem,
                                    s);
        const long long items = (long long)nx * ny * ((nz + kZChunk - 1) / kZChunk);
        const int gz = int(std::max<long long>(1, std::min<long long>((items + kWarps - 1) / kWarps,
                                                                      (long long)device_sms() * 8)));
        launch_conv_z_chunk<C, TO>(reinterpret_cast<const float*>(tmp_a), out, tpz, R[2], nx, ny, nz, gz, s);
        count(2);
        return;
      }
    }
    conv_pass<TI, C>(in, tmp_a, tp[0] ? tp[0] : unit_tap(), R[0], 0, s);
    conv_pass<C, C>(tmp_a, tmp_b, tp[1] ? tp[1] : unit_tap(), R[1], 1, s);
    conv_pass<C, TO>(tmp_b, out, tp[2] ? tp[2] : unit_tap(), R[2], 2, s);
    count(3);
  }

  // One axis pass: VG = 4 z values per thread when nz % 4 == 0.
  template <typename TI, typename TO>
  void conv_pass(const TI* in, TO* out, const C* tp, int r, int axis, cudaStream_t s) {
    const int vg = nz % 4 == 0 ? 4 : 1;
    const int nzg = nz / vg;
    long long nb;
    if (axis < 2) {
      const int na = axis == 0 ? nx : ny, no = axis == 0 ? ny : nx;
      nb = (long long)no * ((na + kConvA - 1) / kConvA) * ((nzg + kConvZ - 1) / kConvZ);
    } else {
      const int lpb = kThreads / std::min(nzg, kThreads);
      nb = ((long long)nx * ny + lpb - 1) / lpb;
    }
    const int grid = int(std::max<long long>(1, std::min<long long>(nb, (long long)device_sms() * 16)));
    if (axis < 2) {
      if (vg == 4)
        k_conv_xy<TI, TO, C, 4><<<grid, kThreads, 0, s>>>(in, out, tp, r, nx, ny, nz, axis);
      else
        k_conv_xy<TI, TO, C, 1><<<grid, kThreads, 0, s>>>(in, out, tp, r, nx, ny, nz, axis);
    } else {
      if (vg == 4)
        k_conv_z<TI, TO, C, 4><<<grid, kThreads, 0, s>>>(in, out, tp, r, nx, ny, nz);
      else
        k_conv_z<TI, TO, C, 1><<<grid, kThreads, 0, s>>>(in, out, tp, r, nx, ny, nz);
    }
  }

  C* unit = nullptr;
  C* unit_tap() {
    if (!unit) {
      unit = dalloc<C>(1);
      const C one = C(1);
      ck(cudaMemcpy(unit, &one, sizeof(C), cudaMemcpyHostToDevice), "unit tap");
    }
    return unit;
  }

  void ensure_temps() {
    if (!t1) {
      t1 = dalloc<C>(V);
      t2 = dalloc<C>(V);
      t3 = dalloc<C>(V);
    }
  }

  // -------------------------------------------------------------- setup
  void setup(const float* fT_src, const float* fL_src, const float* fU_src) override {
    if (psf) {
      // the derivative taps exist for every axis with a PSF; identity axes
      // have no sigma to differentiate
    }
    ck(cudaDeviceSynchronize(), "device sync before setup");
    build_tables();
    fT = dalloc<float>(V);
    ck(cudaMemcpyAsync(fT, fT_src, V * sizeof(float), cudaMemcpyDefault, stream), "copy f_T");
    const int gv = grid_for((long long)V);
    // target statistics
    TargetStats* d_stats = dalloc<TargetStats>(1);
    TargetStats init{0, 0, 0x7f800000u, 0u};
    ck(cudaMemcpyAsync(d_stats, &init, sizeof(init), cudaMemcpyHostToDevice, stream), "stats init");
    k_target_stats<<<gv, kThreads, 0, stream>>>(fT, (long long)V, d_stats);
    TargetStats hs;
    ck(cudaMemcpyAsync(&hs, d_stats, sizeof(hs), cudaMemcpyDeviceToHost, stream), "stats");
    ck(cudaStreamSynchronize(stream), "target stats");
    if (hs.n_bad) fail(SIPO_ERR_INVALID_ARG, "target contains NaN, infinite or negative values");
    if (hs.n_gel == 0) fail(SIPO_ERR_INVALID_ARG, "empty gelation region (target is all zero)");
    // Case 1 with explicit per-voxel bounds f_L <= f_U on gel (the response-
    // domain tolerances of Sec. 2.7.1 mapped through M^-1): f_crit = min f_L
    float* fLd = nullptr;
    float* fUd = nullptr;
    if (fL_src) {
      ck(cudaMallocAsync(reinterpret_cast<void**>(&fLd), V * sizeof(float), stream), "bounds tmp");
      ck(cudaMallocAsync(reinterpret_cast<void**>(&fUd), V * sizeof(float), stream), "bounds tmp");
      ck(cudaMemcpyAsync(fLd, fL_src, V * sizeof(float), cudaMemcpyDefault, stream), "copy f_L");
      ck(cudaMemcpyAsync(fUd, fU_src, V * sizeof(float), cudaMemcpyDefault, stream), "copy f_U");
      TargetStats bs{0, 0, 0x7f800000u, 0u};
      ck(cudaMemcpyAsync(d_stats, &bs, sizeof(bs), cudaMemcpyHostToDevice, stream), "stats init");
      k_bound_stats<<<gv, kThreads, 0, stream>>>(fT, fLd, fUd, (long long)V, d_stats);
      ck(cudaMemcpyAsync(&bs, d_stats, sizeof(bs), cudaMemcpyDeviceToHost, stream), "stats");
      ck(cudaStreamSynchronize(stream), "bound stats");
      if (bs.n_bad) {
        cudaFreeAsync(fLd, stream);
        cudaFreeAsync(fUd, stream);
        cudaStreamSynchronize(stream);
        fail(SIPO_ERR_INVALID_ARG, "explicit bounds need 0 < f_L <= f_U (finite) on every gel voxel");
      }
      hs.min_bits = bs.min_bits;
      hs.max_bits = bs.max_bits;
    }
    float fmin_v, fmax_v;
    std::memcpy(&fmin_v, &hs.min_bits, 4);
    std::memcpy(&fmax_v, &hs.max_bits, 4);
    const double mn = fmin_v;
    // normalisation (Sec. 2.5; Case 1 Eqs. 29-31; Case 2 Eq. 39)
    double mult = 1.0;
    has_u = cp.kase == SIPO_GENERAL || cp.kase == SIPO_CASE1;
    has_v = cp.kase == SIPO_GENERAL || cp.kase == SIPO_CASE2;
    band_rhs = has_u ? 0.0 : 1.0;
    if (cp.kase == SIPO_GENERAL) {
      f_crit = mn;
      mult = 1.0 / f_crit;
      c_u = cp.w1;
      c_v = cp.w2;
    } else if (cp.kase == SIPO_CASE1 && fLd) {
      f_crit = mn;  // min f_L
      mult = 1.0 / f_crit;
      up_ratio = 0.0;
      c_u = 1.0;
      c_v = 0.0;
    } else if (cp.kase == SIPO_CASE1) {
      f_crit = (1.0 - cp.tol_lo) * mn;
      mult = (1.0 - cp.tol_lo) / f_crit;
      up_ratio = (1.0 + cp.tol_hi) / (1.0 - cp.tol_lo);
      c_u = 1.0;
      c_v = 0.0;
    } else {
      f_crit = cp.inhibit_ratio * mn;
      mult = 1.0 / f_crit;
      c_u = 0.0;
      c_v = 1.0;
    }
    ft_is_const = hs.min_bits == hs.max_bits;
    ft_const = C(double(fmin_v) * mult);
    lab = dalloc<uint8_t>(V);
    if (!ft_is_const) {
      ft = dalloc<C>(V);
    }
    // labels
    {
      int *da = nullptr, *db = nullptr;
      uint8_t *ma = nullptr, *mb = nullptr;
      ck(cudaMallocAsync(reinterpret_cast<void**>(&da), V * sizeof(int), stream), "labels tmp");
      ck(cudaMallocAsync(reinterpret_cast<void**>(&db), V * sizeof(int), stream), "labels tmp");
      k_gel_init<<<gv, kThreads, 0, stream>>>(fT, (long long)V, da, lab);
      const int W = cp.band_width;
      const bool band_free = W < 0;
      if (!band_free) {
        k_dist_pass<<<gv, kThreads, 0, stream>>>(da, db, W, nx, ny, nz, 0);
        k_dist_pass<<<gv, kThreads, 0, stream>>>(db, da, W, nx, ny, nz, 1);
        k_dist_pass<<<gv, kThreads, 0, stream>>>(da, db, W, nx, ny, nz, 2);
      }
      uint8_t* sup = nullptr;
      if (psf && !band_free) {
        ck(cudaMallocAsync(reinterpret_cast<void**>(&ma), V, stream), "labels tmp");
        ck(cudaMallocAsync(reinterpret_cast<void**>(&mb), V, stream), "labels tmp");
        k_gel_mask<<<gv, kThreads, 0, stream>>>(lab, ma, (long long)V);
        k_dilate_pass<<<gv, kThreads, 0, stream>>>(ma, mb, R[0], nx, ny, nz, 0);
        k_dilate_pass<<<gv, kThreads, 0, stream>>>(mb, ma, R[1], nx, ny, nz, 1);
        k_dilate_pass<<<gv, kThreads, 0, stream>>>(ma, mb, R[2], nx, ny, nz, 2);
        sup = mb;
      }
      k_labels_final<C><<<gv, kThreads, 0, stream>>>(lab, band_free ? nullptr : db, sup,
                                                      band_free ? -1 : W, band_free ? 1 : 0, geo());
      ck(cudaFreeAsync(da, stream), "free");
      ck(cudaFreeAsync(db, stream), "free");
      if (ma) ck(cudaFreeAsync(ma, stream), "free");
      if (mb) ck(cudaFreeAsync(mb, stream), "free");
    }
    if (!ft_is_const) k_ft<C><<<gv, kThreads, 0, stream>>>(fLd ? fLd : fT, lab, mult, ft, (long long)V);
    if (fLd) {
      fu = dalloc<C>(V);
      k_ft<C><<<gv, kThreads, 0, stream>>>(fUd, lab, mult, fu, (long long)V);
      ck(cudaFreeAsync(fLd, stream), "free");
      ck(cudaFreeAsync(fUd, stream), "free");
      count(2);
    }
    // columns that need the backprojection inside the solve
    need = dalloc<uint8_t>(size_t(nx) * ny);
    {
      const int gc = grid_for((long long)nx * ny);
      if (psf) {
        uint8_t* tmp = nullptr;
        ck(cudaMallocAsync(reinterpret_cast<void**>(&tmp), size_t(nx) * ny, stream), "need tmp");
        k_need_cols<<<gc, kThreads, 0, stream>>>(lab, tmp, nx, ny, nz);
        k_dilate_cols<<<gc, kThreads, 0, stream>>>(tmp, need, nx, ny, R[0], R[1]);
        ck(cudaFreeAsync(tmp, stream), "free");
      } else {
        k_need_cols<<<gc, kThreads, 0, stream>>>(lab, need, nx, ny, nz);
      }
    }
    rspan = dalloc<int2>(size_t(na) * nd);
    launch_ray_spans<C>(geo(), need, rspan, stream);
    {
      const int wr = (nx + 2 * kNbPad + 31) / 32 + 1, wc = (ny + 2 * kNbPad + 31) / 32 + 1;
      uint32_t* br = dalloc<uint32_t>(size_t(ny) * wr);
      uint32_t* bc = dalloc<uint32_t>(size_t(nx) * wc);
      launch_need_bits(need, br, bc, nx, ny, wr, wc, stream);
      nbits.rows = br;
      nbits.cols = bc;
      nbits.wr = wr;
      nbits.wc = wc;
    }
    // iterate storage
    y = dalloc<S>(SN); y0 = dalloc<S>(SN); yp = dalloc<S>(SN); ybar = dalloc<S>(SN);
    gp = dalloc<C>(SN); g0 = dalloc<C>(SN); gc = dalloc<C>(SN); col = dalloc<C>(SN);
    mask = dalloc<uint8_t>(SN);
    act_col = dalloc<uint8_t>(size_t(na) * nd);
    lu = dalloc<S>(V); ll = dalloc<S>(V); lu0 = dalloc<S>(V); ll0 = dalloc<S>(V);
    lpu = dalloc<S>(V); lpl = dalloc<S>(V); q = dalloc<S>(V); qp = dalloc<S>(V);
    d = dalloc<C>(V); d0 = dalloc<C>(V); dp = dalloc<C>(V); row = dalloc<C>(V);
    st = dalloc<Scal>(1);
    part = dalloc<double>(size_t(kNumSlots) * kRedBlocks);
    trace = dalloc<double>(size_t(kTraceCap) * kTraceFields);
    ensure_temps();
    if (psf) kq = dalloc<S>(V);
    // P^T y-bar in the compute type: the PSF path blurs it; the check step of
    // both paths hands it to the element-wise dual update (k_dual), whose FP64
    // check reductions would otherwise spill inside the backprojector
    braw = dalloc<C>(V);
    ck(cudaMemsetAsync(braw, 0, V * sizeof(C), stream), "memset");
    const Geo<C> g = geo();
    const Bufs<S, C> B = bufs();
    // active rays: [P_mu f_T]_j > 0 with the unblurred operator (Sec. 2.2)
    const C* src = nullptr;
    if constexpr (sizeof(C) == 4) {
      src = reinterpret_cast<const C*>(fT);
    } else {
      k_convert<float, C><<<gv, kThreads, 0, stream>>>(fT, t1, (long long)V);
      src = t1;
    }
    launch_project<C, C, C, kFpStore, C>(g, src, Bufs<C, C>{}, gp, nullptr, zl, stream);
    const int gs = grid_for((long long)SN);
    k_mask<C><<<gs, kThreads, 0, stream>>>(gp, mask, g0, (long long)SN);
    k_act_cols<<<grid_for((long long)na * nd), kThreads, 0, stream>>>(mask, act_col, (long long)na * nd, nz);
    // column abs-sums of G: A (1_band + 2 1_gel) on active rays
    k_row_indicator<C><<<gv, kThreads, 0, stream>>>(lab, t1, (long long)V);
    if (psf) {
      psf3<C, C>(t1, t2, t3, braw, -1, stream);
      ck(cudaMemsetAsync(braw, 0, V * sizeof(C), stream), "memset");
      launch_project<C, C, C, kFpStore, C>(g, t2, Bufs<C, C>{}, col, nullptr, zl, stream);
    } else {
      launch_project<C, C, C, kFpStore, C>(g, t1, Bufs<C, C>{}, col, nullptr, zl, stream);
    }
    k_apply_mask<C><<<gs, kThreads, 0, stream>>>(col, mask, (long long)SN);
    // row abs-sums of A^T over active rays: A^T 1_act = K P^T 1_act
    if (psf) {
      launch_backproject<C, C, C, kBpStore, C>(g, g0, Bufs<C, C>{}, t1, nullptr, zl, stream);
      psf3<C, C>(t1, row, t2, t3, -1, stream);
    } else {
      launch_backproject<C, C, C, kBpStore, C>(g, g0, Bufs<C, C>{}, row, nullptr, zl, stream);
    }
    (void)B;
    // setup sums
    k_setup_sums<C><<<kRedBlocks, kThreads, 0, stream>>>(lab, ft_is_const ? nullptr : ft, ft_const, fu, row,
                                                         up_ratio, has_u, has_v, cp.kase, (long long)V, part);
    std::vector<double> hp(8 * size_t(kRedBlocks));
    ck(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, stream), "sums");
    ck(cudaStreamSynchronize(stream), "setup");
    double sums[8] = {};
    for (int i = 0; i < 8; ++i)
      for (int b = 0; b < kRedBlocks; ++b) sums[i] += hp[size_t(i) * kRedBlocks + b];
    fu_sum = fu ? sums[7] : 0.0;
    n_band = (long long)sums[0];
    n_gel = (long long)sums[1];
    if (has_u && c_u != 0.0 && n_band == 0)
      fail(SIPO_ERR_INVALID_ARG,
           "empty band: the band maximum u~ is in no row (band_width 0 without a PSF in Case 1 or the general "
           "form); the LP is unbounded");
    col_u = has_u ? sums[0] : 0.0;
    col_v = has_v ? sums[2] : 0.0;
    h_norm = std::sqrt(sums[0] * band_rhs * band_rhs + (cp.kase == SIPO_CASE1 ? sums[4] : 0.0) + sums[3]);
    c_norm = std::sqrt((has_u ? c_u * c_u : 0.0) + (has_v ? c_v * c_v : 0.0));
    const double c_hat2 = (has_u && col_u > 0 ? c_u * c_u / col_u : 0.0) +
                          (has_v && col_v > 0 ? c_v * c_v / col_v : 0.0);
    const double h_hat2 = sums[5] + sums[6];
    omega0 = (c_hat2 > 0 && h_hat2 > 0) ? std::sqrt(c_hat2 / h_hat2) : 1.0;
    if (tol.primal_weight > 0) omega0 = tol.primal_weight;
    // bound-based infeasibility certificate (Cases 1 and 2): b = A 1_rows and
    // B = sum of the constant upper bounds of those rows
    cert_on = cp.kase == SIPO_CASE1 || cp.kase == SIPO_CASE2;
    if (cert_on) {
      cert_q = dalloc<C>(V);
      cert_b = dalloc<C>(SN);
      k_cert_rows<C><<<gv, kThreads, 0, stream>>>(lab, t1, cp.kase == SIPO_CASE2 ? 2 : 1, (long long)V);
      if (psf) {
        psf3<C, C>(t1, t2, t3, braw, -1, stream);
        ck(cudaMemsetAsync(braw, 0, V * sizeof(C), stream), "memset");
        launch_project<C, C, C, kFpStore, C>(g, t2, Bufs<C, C>{}, cert_b, nullptr, zl, stream);
      } else {
        launch_project<C, C, C, kFpStore, C>(g, t1, Bufs<C, C>{}, cert_b, nullptr, zl, stream);
      }
      cert_B = cp.kase == SIPO_CASE2 ? double(n_band) * band_rhs : (fu ? sums[7] : up_ratio * sums[2]);
      count(3);
      // slice by slice when the operator does not couple z-slices
      cert_slices = R[2] == 0 && nz > 1 && nz <= kCertMaxZ;
      if (cert_slices) {
        cert_Bz = dalloc<double>(size_t(nz));
        cert_pz = dalloc<double>(size_t(kCertBlocks) * nz);
        cert_kz = dalloc<unsigned long long>(size_t(nz));
        k_cert_bz<C><<<kCertBlocks, kThreads, 0, stream>>>(lab, ft_is_const ? nullptr : ft, ft_const, fu,
                                                            up_ratio, cp.kase, (long long)nx * ny, nz, cert_pz);
        k_cert_zsum<<<(nz + kThreads - 1) / kThreads, kThreads, 0, stream>>>(cert_pz, kCertBlocks, nz, cert_Bz);
        zero(cert_kz, size_t(nz));
        count(2);
      }
    }
    count(16);
    choose_tiles();
  }

  // ------------------------------------------------------- iteration steps
  template <typename T>
  void zero(T* p, size_t n) {
    ck(cudaMemsetAsync(p, 0, n * sizeof(T), stream), "memset");
  }

  void begin_solve() override {
    if (!warm_pending) init_state();
    warm_pending = false;
    build_graph();
    launches = 0;
    t_start = std::chrono::steady_clock::now();
  }

  // zero start of a solve (y = 0, lambda = 0, u~ = 0, v~ = 1, omega = omega0)
  void init_state() {
    zero(y, SN); zero(y0, SN); zero(yp, SN); zero(ybar, SN); zero(gp, SN); zero(g0, SN); zero(gc, SN);
    zero(lu, V); zero(ll, V); zero(lu0, V); zero(ll0, V); zero(lpu, V); zero(lpl, V);
    zero(q, V); zero(qp, V); zero(d, V); zero(d0, V); zero(dp, V);
    if (kq) zero(kq, V);
    zero(part, size_t(kNumSlots) * kRedBlocks);
    Scal h{};
    h.c_u = c_u; h.c_v = c_v; h.band_rhs = band_rhs; h.col_u = col_u; h.col_v = col_v;
    h.h_norm = h_norm; h.c_norm = c_norm; h.kkt_tol = tol.kkt_tol; h.has_u = has_u; h.has_v = has_v;
    h.max_iter = tol.max_iter;
    h.u = 0.0; h.v = 1.0; h.u0 = 0.0; h.v0 = 1.0; h.up = 0.0; h.vp = 1.0;
    h.omega = omega0;
    h.trace = trace;
    h.trace_cap = kTraceCap;
    h.trace_n = 0;
    h.cert_B = cert_B;
    h.cert_on = cert_on ? 1 : 0;
    h.cert = 0;
    h.cert_slices = cert_slices ? 1 : 0;
    h.cert_z = -1;
    if (cert_kz) zero(cert_kz, size_t(nz));
    *h_st = h;
    ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
    ck(cudaStreamSynchronize(stream), "begin solve");
    solved = false;
  }

  // Tile table (kBpTiles entries, see launch_backproject).  tile_cfg >= 0
  // selects an entry; -1 times a few un-captured iterations of each entry with
  // CUDA events (backprojection phase) and keeps the fastest.
  void choose_tiles() {
    if (tol.tile_cfg >= 0) {
      if (tol.tile_cfg >= kBpTiles) fail(SIPO_ERR_INVALID_ARG, "tile_cfg out of range");
      bp_nv = tol.tile_cfg;
      return;
    }
    const TileKey key{nx, ny, nz, na, nd, tol.storage, psf ? 1 : 0};
    {
      std::lock_guard<std::mutex> lock(g_tile_mutex);
      auto it = g_tile_cache.find(key);
      if (it != g_tile_cache.end()) {
        bp_nv = it->second;
        return;
      }
    }
    float best = 1e30f;
    int best_tile = 0;
    cudaEvent_t ev[7];
    for (auto& e : ev) ck(cudaEventCreate(&e), "event");
    for (int tile = 0; tile < kBpTiles; ++tile) {
      bp_nv = tile;
      init_state();
      float tot = 0.0f;
      for (int it = 0; it < 4; ++it) {
        enqueue_normal(stream, ev);
        ck(cudaStreamSynchronize(stream), "autotune");
        float t = 0.0f;
        ck(cudaEventElapsedTime(&t, ev[3], ev[6]), "elapsed");
        if (it > 0) tot += t;  // first iteration is a warm-up
      }
      if (tot < best) { best = tot; best_tile = tile; }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    bp_nv = best_tile;
    std::lock_guard<std::mutex> lock(g_tile_mutex);
    g_tile_cache[key] = best_tile;
  }

  void enqueue_psf_q(const S* src, cudaStream_t s) { psf3<S, S>(src, kq, t1, t2, -1, s); }

  void enqueue_normal(cudaStream_t s, cudaEvent_t* ev = nullptr) {
    const Geo<C> g = geo();
    const Bufs<S, C> B = bufs();
    const long long nvv = (long long)(V / ze);
    auto rec = [&](int i) {
      if (ev) ck(cudaEventRecord(ev[i], s), "event");
    };
    rec(0);
    k_scalar_step<false><<<1, kThreads, 0, s>>>(st, part);
    count(1);
    rec(1);
    if (psf) enqueue_psf_q(q, s);
    rec(2);
    launch_project<S, S, C, kFpPrimal, C>(g, psf ? kq : q, B, (C*)nullptr, act_col, zl, s, nbits, rspan);
    count(1);
    rec(3);
    if (psf) {
      launch_backproject<S, S, C, kBpStore, C>(g, ybar, B, braw, need, zl, s, bp_nv);
      count(1);
      rec(4);
      psf3<C, C>(braw, t3, t1, t2, -1, s);
      rec(5);
      dual_launch<false>(B, t3, nvv, s);
    } else {
      launch_backproject<S, S, C, kBpDual, C>(g, ybar, B, (C*)nullptr, need, zl, s, bp_nv);
      count(1);
      rec(4);
      rec(5);
    }
    rec(6);
  }

  template <bool CHECK>
  void dual_launch(const Bufs<S, C>& B, const C* dbar, long long nvv, cudaStream_t s) {
    if (ze > 1)
      k_dual<S, C, z_group<C>(), CHECK><<<kRedBlocks, kThreads, 0, s>>>(B, dbar, nvv);
    else
      k_dual<S, C, 1, CHECK><<<kRedBlocks, kThreads, 0, s>>>(B, dbar, nvv);
    count(1);
  }

  void enqueue_check(cudaStream_t s) {
    const Geo<C> g = geo();
    const Bufs<S, C> B = bufs();
    const long long nvv = (long long)(V / ze), nvs = (long long)(SN / ze);
    k_scalar_step<true><<<1, kThreads, 0, s>>>(st, part);
    count(1);
    if (psf) enqueue_psf_q(q, s);
    launch_project<S, S, C, kFpPrimalCheck, C>(g, psf ? kq : q, B, (C*)nullptr, act_col, zl, s, nbits, rspan);
    count(1);
    if (psf) {
      launch_backproject<S, S, C, kBpStore, C>(g, ybar, B, braw, need, zl, s, bp_nv);
      count(1);
      psf3<C, C>(braw, t3, t1, t2, -1, s);
      dual_launch<true>(B, t3, nvv, s);
      enqueue_psf_q(qp, s);
    } else {
      launch_backproject<S, S, C, kBpStore, C>(g, ybar, B, braw, need, zl, s, bp_nv);
      count(1);
      dual_launch<true>(B, braw, nvv, s);
    }
    launch_project<S, S, C, kFpResid, C>(g, psf ? kq : qp, B, (C*)nullptr, act_col, zl, s, nbits, rspan);
    count(1);
    enqueue_certificate(s);
    k_scalar_check<<<1, kThreads, 0, s>>>(st, part);
    count(1);
    if (ze > 1) {
      k_blend_sino<S, C, z_group<C>()><<<grid_for(nvs), kThreads, 0, s>>>(B, nvs);
      k_blend_vol<S, C, z_group<C>()><<<kRedBlocks, kThreads, 0, s>>>(B, nvv);
    } else {
      k_blend_sino<S, C, 1><<<grid_for(nvs), kThreads, 0, s>>>(B, nvs);
      k_blend_vol<S, C, 1><<<kRedBlocks, kThreads, 0, s>>>(B, nvv);
    }
    count(2);
  }

  // Bound-based certificate of the epoch difference lam+ - lam0 (per slice when
  // the operator does not couple z-slices): sets st->cert (and st->cert_z).
  void enqueue_certificate(cudaStream_t s) {
    const Geo<C> g = geo();
    const Bufs<S, C> B = bufs();
    if (cert_slices) {
      k_cert_vol_z<S, C><<<kCertBlocks, kThreads, 0, s>>>(B, (long long)nx * ny, nz, cert_pz);
      const C* cq = cert_q;
      if (psf) {
        psf3<C, C>(cert_q, t3, t1, t2, -1, s);
        cq = t3;
      }
      launch_project<C, S, C, kFpCertZ, C>(g, cq, B, (C*)nullptr, act_col, zl, s, nbits, rspan);
      k_cert_decide_z<<<1, kThreads, 0, s>>>(st, cert_pz, kCertBlocks, nz, cert_kz, cert_Bz);
      count(3);
    } else if (cert_on) {
      k_cert_vol<S, C><<<kRedBlocks, kThreads, 0, s>>>(B, (long long)V);
      const C* cq = cert_q;
      if (psf) {
        psf3<C, C>(cert_q, t3, t1, t2, -1, s);
        cq = t3;
      }
      launch_project<C, S, C, kFpCert, C>(g, cq, B, (C*)nullptr, act_col, zl, s, nbits, rspan);
      k_cert_decide<<<1, kThreads, 0, s>>>(st, part);
      count(3);
    }
  }

  void build_graph() {
    if (gexec) return;
    cudaGraph_t graph;
    const long long before = launches;
    ck(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    enqueue_check(stream);
    for (int i = 1; i < P; ++i) enqueue_normal(stream);
    cudaError_t e = cudaStreamEndCapture(stream, &graph);
    ck(e, "end capture");
    graph_nodes = launches - before;
    launches = before;
    g_launches -= graph_nodes;
    ck(cudaGraphInstantiate(&gexec, graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
  }

  void launch_block(long long n) override {
    if (n == P) {
      build_graph();
      ck(cudaGraphLaunch(gexec, stream), "graph launch");
      count(graph_nodes);
    } else {
      enqueue_check(stream);
      for (long long i = 1; i < n; ++i) enqueue_normal(stream);
    }
    ck(cudaGetLastError(), "launch");
  }

  void stop_at_last_check() override {
    ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, stream), "read state");
    ck(cudaStreamSynchronize(stream), "stop");
    if (!h_st->done) {
      h_st->done = 1;
      h_st->status = SIPO_ITER_LIMIT;
      ck(cudaMemcpyAsync(st, h_st, sizeof(Scal), cudaMemcpyHostToDevice, stream), "state");
      ck(cudaStreamSynchronize(stream), "stop");
    }
  }

  void request_done() override {
    ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, stream), "read state");
  }

  bool done_flag() override {
    ck(cudaStreamSynchronize(stream), "iterations");
    return h_st->done != 0;
  }

  void final_check() {
    enqueue_check(stream);
    ck(cudaGetLastError(), "launch");
  }

  void finish_solve(void* y_out, int loc, sipo_result* res) override {
    ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, stream), "read state");
    ck(cudaStreamSynchronize(stream), "solve");
    check_bp_fault();
    if (!h_st->done) {
      final_check();
      ck(cudaMemcpyAsync(h_st, st, sizeof(Scal), cudaMemcpyDeviceToHost, stream), "read state");
      ck(cudaStreamSynchronize(stream), "solve");
    }
    solved = true;
    if (h_st->numeric)
      fail(SIPO_ERR_NUMERIC, "solve stopped at iteration " + std::to_string(h_st->k) +
                                 ": non-finite residuals or objectives (NaN or infinite iterates)");
    // f~* = A^T y* of the returned point, recomputed by one plain application
    // of the operator: the iterations carry d by linearity (d+ = (d_bar + d) / 2),
    // which drifts from A^T y by rounding over many steps in FP32
    launch_backproject<S, S, C, kBpStore, C>(geo(), yp, bufs(), psf ? braw : dp, need, zl, stream, bp_nv);
    count(1);
    if (psf) psf3<C, C>(braw, dp, t1, t2, -1, stream);
    // metrics of d = A^T y at the returned point (Eqs. 6-8, 27, 46)
    k_metrics<C><<<kRedBlocks, kThreads, 0, stream>>>(dp, lab, fT, ft_is_const ? nullptr : ft, ft_const,
                                                     f_crit, (long long)V, part);
    count(1);
    std::vector<double> hp(8 * size_t(kRedBlocks));
    ck(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, stream), "metrics");
    if (y_out) copy_out(yp, SN, y_out, loc, conv_tmp(SN));
    ck(cudaStreamSynchronize(stream), "metrics");
    double m[8] = {1e300, -1e300, -1e300, 1e300, 0.0, 0.0, 1e300, -1e300};
    for (int b = 0; b < kRedBlocks; ++b) {
      m[0] = std::min(m[0], hp[0 * kRedBlocks + b]);
      m[1] = std::max(m[1], hp[1 * kRedBlocks + b]);
      m[2] = std::max(m[2], hp[2 * kRedBlocks + b]);
      m[3] = std::min(m[3], hp[3 * kRedBlocks + b]);
      m[4] += hp[4 * kRedBlocks + b];
      m[5] += hp[5 * kRedBlocks + b];
      m[6] = std::min(m[6], hp[6 * kRedBlocks + b]);
      m[7] = std::max(m[7], hp[7 * kRedBlocks + b]);
    }
    const Scal& h = *h_st;
    std::memset(res, 0, sizeof(*res));
    // a solve stopped by its caller before a decision (a probe's certificate)
    // reports the iteration limit
    res->status = h.done ? h.status : SIPO_ITER_LIMIT;
    res->restarts = h.restarts;
    res->iters = h.k;
    res->kkt = h.kkt; res->rel_primal = h.rel_p; res->rel_dual = h.rel_d; res->rel_gap = h.rel_gap;
    res->r_primal = h.rp; res->r_dual = h.rd; res->gap = h.gap; res->pobj = h.pobj; res->dobj = h.dobj;
    res->u = h.up; res->v = h.vp; res->omega = h.omega;
    res->f_crit = f_crit;
    res->dtvr_f = m[0] > 0 ? m[1] / m[0] : INFINITY;
    res->dsr = (m[0] > 0 && n_band > 0) ? m[2] / m[0] : INFINITY;
    res->psr_f = (n_band > 0 && m[2] > 0) ? m[3] / m[2] : INFINITY;
    res->alpha = m[5] > 0 ? m[4] / m[5] : 0.0;
    res->s = m[6];
    res->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    res->kernel_launches = launches;
    res->tile_cfg = bp_nv;
    res->cert_slice = h.status == 1 ? h.cert_z : -1;
  }

  // A bounded wait inside the staged backprojector gave up (bit 0), or an
  // angle's rows did not fit its box (bit 1): the sums of that launch are not
  // valid, so the solve is an error.
  void check_bp_fault() {
    const unsigned int f = bp3_fault_take();
    if (f & 1u) fail(SIPO_ERR_TIMEOUT, "backprojector: a wait on a tensor-memory copy timed out");
    if (f) fail(SIPO_ERR_NUMERIC, "backprojector: detector rows outside the staged box");
  }

  // copies n elements of S (converted to C) to out (host or device)
  template <typename T>
  void copy_out(const T* src, size_t n, void* out, int loc, C* tmp) {
    const C* from;
    if constexpr (std::is_same<T, C>::value) {
      from = src;
    } else {
      k_convert<T, C><<<grid_for((long long)n), kThreads, 0, stream>>>(src, tmp, (long long)n);
      count(1);
      from = tmp;
    }
    ck(cudaMemcpyAsync(out, from, n * sizeof(C), loc == SIPO_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice,
                       stream), "copy out");
  }

  // ------------------------------------------------------------ operators
  void project(const void* vol, void* sino, cudaStream_t s) override {
    const Geo<C> g = geo();
    const C* src = static_cast<const C*>(vol);
    if (psf) {
      ensure_temps();
      psf3<C, C>(src, t3, t1, t2, -1, s);
      src = t3;
    }
    launch_project<C, C, C, kFpStore, C>(g, src, Bufs<C, C>{}, static_cast<C*>(sino), nullptr, zl, s);
    count(1);
    ck(cudaGetLastError(), "project");
  }

  void backproject(const void* sino, void* vol, cudaStream_t s) override {
    const Geo<C> g = geo();
    if (psf) {
      ensure_temps();
      launch_backproject<C, C, C, kBpStore, C>(g, static_cast<const C*>(sino), Bufs<C, C>{}, t3, nullptr, zl, s,
                                               bp_nv);
      psf3<C, C>(t3, static_cast<C*>(vol), t1, t2, -1, s);
    } else {
      launch_backproject<C, C, C, kBpStore, C>(g, static_cast<const C*>(sino), Bufs<C, C>{},
                                               static_cast<C*>(vol), nullptr, zl, s, bp_nv);
    }
    count(1);
    ck(cudaGetLastError(), "backproject");
  }

  void psf_apply(const void* in, void* out, int deriv, cudaStream_t s) override {
    ensure_temps();
    if (deriv >= 0 && R[deriv] == 0) {
      ck(cudaMemsetAsync(out, 0, V * sizeof(C), s), "memset");
      return;
    }
    psf3<C, C>(static_cast<const C*>(in), static_cast<C*>(out), t1, t2, deriv, s);
    ck(cudaGetLastError(), "psf");
  }

  void psf_grad(const void* sino, const void* vol, double* grad, cudaStream_t s) override {
    ensure_temps();
    if (!tvol) tvol = dalloc<C>(V);
    std::vector<double> hp(kRedBlocks);
    double* pg = dalloc_part();
    // b = P_mu^T sino, recomputed (not stored by the forward pass)
    launch_backproject<C, C, C, kBpStore, C>(geo(), static_cast<const C*>(sino), Bufs<C, C>{}, tvol, nullptr,
                                             zl, s);
    count(1);
    for (int a = 0; a < 3; ++a) {
      grad[a] = 0.0;
      if (R[a] == 0) continue;
      psf3<C, C>(static_cast<const C*>(vol), t3, t1, t2, a, s);
      k_dot<C><<<kRedBlocks, kThreads, 0, s>>>(tvol, t3, (long long)V, pg);
      count(1);
      ck(cudaMemcpyAsync(hp.data(), pg, kRedBlocks * sizeof(double), cudaMemcpyDeviceToHost, s), "grad");
      ck(cudaStreamSynchronize(s), "psf grad");
      for (int i = 0; i < kRedBlocks; ++i) grad[a] += hp[i];
    }
  }

  double* gpart = nullptr;
  double* dalloc_part() {
    if (!gpart) gpart = dalloc<double>(kRedBlocks);
    return gpart;
  }

  void set_sigma(const double* sig) override {
    for (int a = 0; a < 3; ++a) {
      if ((R[a] == 0) != (sig[a] <= 0)) fail(SIPO_ERR_INVALID_ARG, "sigma must stay zero/non-zero per axis");
      sigma[a] = sig[a];
    }
    ck(cudaStreamSynchronize(stream), "sync");
    upload_taps();
  }

  void get_array(int which, void* out, int loc) override {
    const cudaMemcpyKind kind = loc == SIPO_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (which == 0) {
      ck(cudaMemcpyAsync(out, lab, V, kind, stream), "labels");
    } else if (which == 1) {
      ck(cudaMemcpyAsync(out, mask, SN, kind, stream), "mask");
    } else if (which == 2) {
      copy_out(solved ? yp : y, SN, out, loc, conv_tmp(SN));
    } else if (which == 3 || which == 4) {
      copy_out(which == 3 ? (solved ? lpu : lu) : (solved ? lpl : ll), V, out, loc, conv_tmp(V));
    } else if (which == 5) {
      copy_out(solved ? dp : d, V, out, loc, conv_tmp(V));
    } else {
      fail(SIPO_ERR_INVALID_ARG, "unknown array id");
    }
    ck(cudaStreamSynchronize(stream), "get array");
  }

  void profile(int iters, double* ms, int n) override {
    init_state();
    std::vector<cudaEvent_t> ev(7);
    for (auto& e : ev) ck(cudaEventCreate(&e), "event");
    std::vector<double> acc(kNumPhases, 0.0);
    for (int it = 0; it < iters; ++it) {
      enqueue_normal(stream, ev.data());
      ck(cudaStreamSynchronize(stream), "profile");
      for (int i = 0; i < 6; ++i) {
        float t = 0;
        ck(cudaEventElapsedTime(&t, ev[i], ev[i + 1]), "elapsed");
        acc[i] += t;
      }
    }
    // one check step, timed as a whole
    ck(cudaEventRecord(ev[0], stream), "event");
    enqueue_check(stream);
    ck(cudaEventRecord(ev[1], stream), "event");
    ck(cudaStreamSynchronize(stream), "profile");
    float tc = 0;
    ck(cudaEventElapsedTime(&tc, ev[0], ev[1]), "elapsed");
    for (auto& e : ev) cudaEventDestroy(e);
    for (int i = 0; i < std::min(n, kNumPhases); ++i)
      ms[i] = i < 6 ? (iters > 0 ? acc[i] / iters : 0.0) : double(tc);
  }
};

struct Ctx {
  std::unique_ptr<SolverBase> s;
};

int set_error(const Error& e) {
  g_err = e.msg;
  return e.code;
}

}  // namespace

void set_last_error(const std::string& msg) { g_err = msg; }

}  // namespace sipo

struct sipo_ctx {
  sipo::Ctx c;
};

using sipo::Error;

#define SIPO_TRY try {
#define SIPO_CATCH                                       \
  }                                                      \
  catch (const Error& e) { return sipo::set_error(e); } \
  catch (const std::bad_alloc&) {                        \
    sipo::g_err = "host allocation failed";              \
    return SIPO_ERR_OOM;                                 \
  }

extern "C" {

const char* sipo_last_error(void) { return sipo::g_err.c_str(); }

long long sipo_kernel_launch_count(void) { return sipo::g_launches.load(); }

int sipo_phase_count(void) { return sipo::kNumPhases; }

const char* sipo_phase_name(int i) {
  return (i >= 0 && i < sipo::kNumPhases) ? sipo::kPhaseNames[i] : "";
}

int sipo_tile_count(void) { return sipo::kBpTiles; }

unsigned int sipo_check_flags(void) {
#ifdef SIPO_CHECKED
  unsigned int v = 0, zero = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return 0x80000000u;
  if (cudaMemcpyFromSymbol(&v, sipo::g_sipo_check, sizeof(v)) == cudaSuccess)
    cudaMemcpyToSymbol(sipo::g_sipo_check, &zero, sizeof(zero));
  return v | sipo::check_flags_project() | sipo::check_flags_backproject() | 0x40000000u;
#else
  return 0u;
#endif
}

int sipo_wait_selftest(long long budget_cycles, int arrive, int threads, unsigned int* timed_out) {
  SIPO_TRY
  if (!timed_out || budget_cycles <= 0 || threads < 1 || threads > 1024)
    sipo::fail(SIPO_ERR_INVALID_ARG, "wait self-test: null output, budget <= 0 or threads outside 1..1024");
  *timed_out = 0;
  if (sipo::wait_selftest(budget_cycles, arrive, threads, timed_out) != 0)
    sipo::fail(SIPO_ERR_CUDA, "wait self-test: CUDA error");
  if (*timed_out == (unsigned int)threads) {
    sipo::g_err = "wait self-test: every bounded wait gave up";
    return SIPO_ERR_TIMEOUT;
  }
  if (*timed_out != 0) sipo::fail(SIPO_ERR_CUDA, "wait self-test: only some of the waits gave up");
  return SIPO_OK;
  SIPO_CATCH
}

static void create_impl(const sipo_geometry* geo, const float* f_T, const float* f_L, const float* f_U,
                        const sipo_case_params* cp, const sipo_tolerances* tol, void* stream, sipo_ctx** out) {
  sipo::g_err.clear();
  if (!geo || !f_T || !cp || !tol || !out) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (geo->nx <= 0 || geo->ny <= 0 || geo->nz <= 0 || geo->n_angles <= 0 || geo->n_det <= 0 || !geo->angles)
    sipo::fail(SIPO_ERR_INVALID_ARG, "geometry sizes must be positive and angles non-null");
  if ((long long)geo->nx * geo->ny * geo->nz > (1LL << 34) ||
      (long long)geo->n_angles * geo->n_det * geo->nz > (1LL << 34))
    sipo::fail(SIPO_ERR_INVALID_ARG, "problem too large");
  for (int k = 0; k < geo->n_angles; ++k)
    if (!std::isfinite(geo->angles[k])) sipo::fail(SIPO_ERR_INVALID_ARG, "non-finite angle");
  if (geo->mu != 0.0 && !(geo->vial_radius > 0)) sipo::fail(SIPO_ERR_INVALID_ARG, "attenuation needs a vial radius");
  if (!std::isfinite(geo->mu) || geo->mu < 0) sipo::fail(SIPO_ERR_INVALID_ARG, "mu must be finite and >= 0");
  for (int a = 0; a < 3; ++a)
    if (!(geo->psf_sigma[a] >= 0) || geo->psf_sigma[a] > 64) sipo::fail(SIPO_ERR_INVALID_ARG, "psf sigma out of range");
  if (cp->kase < SIPO_GENERAL || cp->kase > SIPO_CASE2) sipo::fail(SIPO_ERR_INVALID_ARG, "unknown LP case");
  if (cp->kase == SIPO_GENERAL && (!(cp->w1 >= 0) || !(cp->w2 >= 0) || !std::isfinite(cp->w1) ||
                                   !std::isfinite(cp->w2)))
    sipo::fail(SIPO_ERR_INVALID_ARG, "weights must be finite and >= 0");
  if (cp->kase == SIPO_CASE1 && (!(cp->tol_lo >= 0 && cp->tol_lo < 1) || !(cp->tol_hi >= 0) ||
                                 !std::isfinite(cp->tol_hi)))
    sipo::fail(SIPO_ERR_INVALID_ARG, "Case 1 tolerances must satisfy 0 <= tol_lo < 1, 0 <= tol_hi < inf");
  if (cp->kase == SIPO_CASE2 && !(cp->inhibit_ratio > 0 && std::isfinite(cp->inhibit_ratio)))
    sipo::fail(SIPO_ERR_INVALID_ARG, "inhibit_ratio must be finite and > 0");
  if (cp->band_width > 1000) sipo::fail(SIPO_ERR_INVALID_ARG, "band_width too large");
  if (tol->storage != SIPO_F32 && tol->storage != SIPO_F64 && tol->storage != SIPO_BF16)
    sipo::fail(SIPO_ERR_INVALID_ARG, "unknown storage type");
  if (!(tol->kkt_tol >= 0) || tol->max_iter < 0) sipo::fail(SIPO_ERR_INVALID_ARG, "bad tolerances");
  std::unique_ptr<sipo::SolverBase> s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (tol->storage == SIPO_F32) s.reset(new sipo::Solver<float>(geo, cp, tol, st));
  else if (tol->storage == SIPO_F64) s.reset(new sipo::Solver<double>(geo, cp, tol, st));
  else s.reset(new sipo::Solver<__nv_bfloat16>(geo, cp, tol, st));
  s->setup(f_T, f_L, f_U);
  sipo_ctx* c = new sipo_ctx;
  c->c.s = std::move(s);
  *out = c;
}

int sipo_create(const sipo_geometry* geo, const float* f_T, int f_T_location, const sipo_case_params* cp,
                const sipo_tolerances* tol, void* stream, sipo_ctx** out) {
  SIPO_TRY
  (void)f_T_location;
  create_impl(geo, f_T, nullptr, nullptr, cp, tol, stream, out);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_create_bounded(const sipo_geometry* geo, const float* f_T, const float* f_L, const float* f_U,
                        int location, const sipo_case_params* cp, const sipo_tolerances* tol, void* stream,
                        sipo_ctx** out) {
  SIPO_TRY
  (void)location;
  if (!f_L || !f_U || !cp) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (cp->kase != SIPO_CASE1) sipo::fail(SIPO_ERR_INVALID_ARG, "explicit bounds are a Case-1 form");
  create_impl(geo, f_T, f_L, f_U, cp, tol, stream, out);
  return SIPO_OK;
  SIPO_CATCH
}

static void run_solve(sipo::SolverBase* s) {
  s->begin_solve();
  const long long P = s->period(), M = s->max_iter();
  long long k = 0;
  while (k < M) {
    const long long n = std::min(P, M - k);
    s->launch_block(n);
    k += n;
    s->request_done();
    if (s->done_flag()) break;
  }
}

// run_solve that, every `probe_every` iterations (rounded up to check periods)
// and when the solve stops, tests the last check's dual point as a Farkas ray
// of `target`'s LP; stops at the first certificate (sipo_schedule.h).
static void run_solve_probe(sipo::SolverBase* s, sipo::SolverBase* target, long long probe_every, int* certified,
                            int* slice) {
  sipo::probe_schedule(*s, static_cast<sipo::SolverBase*>(nullptr), probe_every,
                       [&](int* sl) { return target->farkas_from(*s, sl) != 0; }, certified, slice);
}

int sipo_solve_probe(sipo_ctx* ctx, sipo_ctx* target, long long probe_every, sipo_result* res, int* certified,
                     int* slice) {
  SIPO_TRY
  if (!ctx || !target || !res || !certified || !slice) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (ctx == target) sipo::fail(SIPO_ERR_INVALID_ARG, "probe: the solved and the tested context are the same");
  if (probe_every <= 0) sipo::fail(SIPO_ERR_INVALID_ARG, "probe_every must be positive");
  target->c.s->farkas_compatible(*ctx->c.s);  // refused before any iteration runs
  run_solve_probe(ctx->c.s.get(), target->c.s.get(), probe_every, certified, slice);
  ctx->c.s->finish_solve(nullptr, SIPO_DEVICE, res);
  return SIPO_OK;
  SIPO_CATCH
}

// run_solve_probe of s with a second solve, `rival`, advanced on its own
// stream at the same time: each round launches one check period of every
// context still running, then reads both states (sipo_schedule.h).
static void run_solve_race(sipo::SolverBase* s, sipo::SolverBase* target, sipo::SolverBase* rival,
                           long long probe_every, int* certified, int* slice) {
  sipo::probe_schedule(*s, rival, probe_every, [&](int* sl) { return target->farkas_from(*s, sl) != 0; },
                       certified, slice);
}

int sipo_solve_race(sipo_ctx* ctx, sipo_ctx* target, sipo_ctx* rival, long long probe_every, sipo_result* res,
                    sipo_result* rival_res, int* certified, int* slice) {
  SIPO_TRY
  if (!ctx || !target || !rival || !res || !rival_res || !certified || !slice)
    sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (ctx == target || ctx == rival || target == rival)
    sipo::fail(SIPO_ERR_INVALID_ARG, "race: the solved, the tested and the rival context must be distinct");
  if (probe_every <= 0) sipo::fail(SIPO_ERR_INVALID_ARG, "probe_every must be positive");
  if (ctx->c.s->dev() != rival->c.s->dev())
    sipo::fail(SIPO_ERR_INVALID_ARG, "race: the solved and the rival context are on different devices");
  target->c.s->farkas_compatible(*ctx->c.s);
  run_solve_race(ctx->c.s.get(), target->c.s.get(), rival->c.s.get(), probe_every, certified, slice);
  ctx->c.s->finish_solve(nullptr, SIPO_DEVICE, res);
  rival->c.s->finish_solve(nullptr, SIPO_DEVICE, rival_res);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_solve(sipo_ctx* ctx, void* y_out, int y_location, sipo_result* res) {
  SIPO_TRY
  if (!ctx || !res) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  run_solve(ctx->c.s.get());
  ctx->c.s->finish_solve(y_out, y_location, res);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_warm_start(sipo_ctx* dst, const sipo_ctx* src) {
  SIPO_TRY
  if (!dst || !src) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (dst == src) sipo::fail(SIPO_ERR_INVALID_ARG, "warm start: source and destination are the same context");
  dst->c.s->warm_from(*src->c.s);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_get_state(sipo_ctx* ctx, void* y, void* lam_up, void* lam_lo, int location, double* scalars) {
  SIPO_TRY
  if (!ctx) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (location != SIPO_HOST && location != SIPO_DEVICE) sipo::fail(SIPO_ERR_INVALID_ARG, "bad location");
  ctx->c.s->state_to(y, lam_up, lam_lo, location, scalars);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_set_state(sipo_ctx* ctx, const void* y, const void* lam_up, const void* lam_lo, int location,
                   const double* scalars) {
  SIPO_TRY
  if (!ctx || !y || !lam_up || !lam_lo || !scalars) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (location != SIPO_HOST && location != SIPO_DEVICE) sipo::fail(SIPO_ERR_INVALID_ARG, "bad location");
  ctx->c.s->state_from(y, lam_up, lam_lo, location, scalars[0], scalars[1], scalars[2]);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_set_primal_from(sipo_ctx* dst, const sipo_ctx* src, double scale, double u, double v) {
  SIPO_TRY
  if (!dst || !src) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (dst == src) sipo::fail(SIPO_ERR_INVALID_ARG, "primal transfer: source and destination are the same context");
  if (!(scale > 0) || !std::isfinite(scale)) sipo::fail(SIPO_ERR_INVALID_ARG, "scale must be finite and > 0");
  dst->c.s->primal_from(*src->c.s, scale, u, v);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_farkas_from(sipo_ctx* ctx, const sipo_ctx* src, int* certified, int* slice) {
  SIPO_TRY
  if (!ctx || !src || !certified) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (ctx == src) sipo::fail(SIPO_ERR_INVALID_ARG, "Farkas test: source and destination are the same context");
  *certified = ctx->c.s->farkas_from(*src->c.s, slice);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_set_primal(sipo_ctx* ctx, const void* y, int y_location, double u, double v) {
  SIPO_TRY
  if (!ctx || !y) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (y_location != SIPO_HOST && y_location != SIPO_DEVICE) sipo::fail(SIPO_ERR_INVALID_ARG, "bad location");
  ctx->c.s->state_from(y, nullptr, nullptr, y_location, u, v, -1.0);
  return SIPO_OK;
  SIPO_CATCH
}

static sipo::Richards richards_of(const sipo_response* M) {
  if (!M) sipo::fail(SIPO_ERR_INVALID_ARG, "null response model");
  if (!(std::isfinite(M->alpha) && std::isfinite(M->k) && std::isfinite(M->f0) && M->k > M->alpha &&
        M->beta > 0 && std::isfinite(M->beta) && M->gamma > 0 && std::isfinite(M->gamma)))
    sipo::fail(SIPO_ERR_INVALID_ARG, "response model needs finite alpha < k, beta > 0, gamma > 0");
  return sipo::Richards{M->alpha, M->k, M->beta, M->gamma, M->f0};
}

int sipo_response_map(const sipo_response* M, const float* in, float* out, long long n, double scale, int inverse,
                      void* stream) {
  SIPO_TRY
  const sipo::Richards r = richards_of(M);
  if (n < 0 || (n > 0 && (!in || !out))) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (!std::isfinite(scale)) sipo::fail(SIPO_ERR_INVALID_ARG, "scale must be finite");
  if (n == 0) return SIPO_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned long long* d_bad = nullptr;
  unsigned long long h_bad = 0;
  sipo::ck(cudaMallocAsync(reinterpret_cast<void**>(&d_bad), sizeof(*d_bad), s), "response map");
  sipo::ck(cudaMemsetAsync(d_bad, 0, sizeof(*d_bad), s), "response map");
  sipo::k_response_map<<<sipo::grid_for(n), sipo::kThreads, 0, s>>>(in, out, n, r, scale, inverse ? 1 : 0, d_bad);
  sipo::ck(cudaGetLastError(), "response map");
  ++sipo::g_launches;
  sipo::ck(cudaMemcpyAsync(&h_bad, d_bad, sizeof(h_bad), cudaMemcpyDeviceToHost, s), "response map");
  sipo::ck(cudaFreeAsync(d_bad, s), "response map");
  sipo::ck(cudaStreamSynchronize(s), "response map");
  if (h_bad) sipo::fail(SIPO_ERR_INVALID_ARG, "response outside the invertible range (>= k, or NaN)");
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_response_inhibit_ratio(const sipo_response* M, const float* m_T, long long n, double m_crit,
                                double* ratio, double* gel_min, void* stream) {
  SIPO_TRY
  const sipo::Richards r = richards_of(M);
  if (!m_T || !ratio || n <= 0) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument or empty target");
  if (!(m_crit > M->alpha && m_crit < M->k)) sipo::fail(SIPO_ERR_INVALID_ARG, "m_crit must lie in (alpha, k)");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned int* d_min = nullptr;
  double* d_out = nullptr;
  sipo::ck(cudaMallocAsync(reinterpret_cast<void**>(&d_min), sizeof(unsigned int), s), "response ratio");
  sipo::ck(cudaMallocAsync(reinterpret_cast<void**>(&d_out), 2 * sizeof(double), s), "response ratio");
  sipo::ck(cudaMemsetAsync(d_min, 0xff, sizeof(unsigned int), s), "response ratio");
  sipo::k_response_gel_min<<<sipo::grid_for(n), sipo::kThreads, 0, s>>>(m_T, n, M->alpha, d_min);
  sipo::k_response_case2_ratio<<<1, 32, 0, s>>>(d_min, r, m_crit, d_out, d_out + 1);
  sipo::ck(cudaGetLastError(), "response ratio");
  sipo::g_launches += 2;
  double h[2];
  sipo::ck(cudaMemcpyAsync(h, d_out, sizeof(h), cudaMemcpyDeviceToHost, s), "response ratio");
  sipo::ck(cudaFreeAsync(d_min, s), "response ratio");
  sipo::ck(cudaFreeAsync(d_out, s), "response ratio");
  sipo::ck(cudaStreamSynchronize(s), "response ratio");
  if (!std::isfinite(h[0])) sipo::fail(SIPO_ERR_INVALID_ARG, "no prescribed response inside (alpha, k)");
  *ratio = h[0];
  if (gel_min) *gel_min = h[1];
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_response_metrics(sipo_ctx* ctx, const sipo_response* M, const float* m_T, int location, double alpha,
                          sipo_response_result* out) {
  SIPO_TRY
  (void)location;
  const sipo::Richards r = richards_of(M);
  if (!ctx || !m_T || !out) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  ctx->c.s->response_metrics(r, m_T, std::isfinite(alpha) ? alpha : 0.0, out);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_solve_batched(sipo_ctx** ctxs, int n, void** y_outs, int y_location, sipo_result* results) {
  SIPO_TRY
  if (!ctxs || n < 0 || (n > 0 && !results)) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  if (n == 0) return SIPO_OK;
  std::vector<sipo::SolverBase*> s(n);
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) sipo::fail(SIPO_ERR_INVALID_ARG, "null context");
    s[i] = ctxs[i]->c.s.get();
    for (int j = 0; j < i; ++j)
      if (s[j] == s[i]) sipo::fail(SIPO_ERR_INVALID_ARG, "a context appears twice in the batch");
    if (s[i]->dev() != s[0]->dev())
      sipo::fail(SIPO_ERR_INVALID_ARG, "the contexts of a batch must have been created on one device");
  }
  for (auto* x : s) x->init_for_batch();
  // One graph per check period of the unfinished contexts: every context's
  // period is a branch forked from, and joined back into, a master stream.
  // The graph is rebuilt without a context once it has finished, so finished
  // contexts launch nothing.
  cudaStream_t master = nullptr;
  sipo::ck(cudaStreamCreateWithFlags(&master, cudaStreamNonBlocking), "stream");
  std::vector<cudaEvent_t> ev(n + 1, nullptr);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto drop_graph = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  };
  auto cleanup = [&]() {
    drop_graph();
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    if (master) cudaStreamDestroy(master);
  };
  try {
    for (auto& e : ev) sipo::ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
    // iteration limits round up to whole check periods; a context whose limit
    // is reached stops at the check that opens its next period
    long long max_periods = 0;
    for (auto* x : s) max_periods = std::max(max_periods, (x->max_iter() + x->period() - 1) / x->period() + 1);
    std::vector<int> live(n);
    for (int i = 0; i < n; ++i) live[i] = i;
    std::vector<long long> per(n, 0);
    for (long long p = 0; p < max_periods && !live.empty(); ++p) {
      if (!exec) {
        sipo::ck(cudaStreamBeginCapture(master, cudaStreamCaptureModeThreadLocal), "begin capture");
        sipo::ck(cudaEventRecord(ev[n], master), "fork");
        for (int i : live) {
          cudaStream_t si = s[i]->strm();
          sipo::ck(cudaStreamWaitEvent(si, ev[n], 0), "fork wait");
          per[i] = s[i]->enqueue_period(si);
          sipo::ck(cudaEventRecord(ev[i], si), "join");
          sipo::ck(cudaStreamWaitEvent(master, ev[i], 0), "join wait");
        }
        sipo::ck(cudaStreamEndCapture(master, &graph), "end capture");
        sipo::ck(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
      }
      sipo::ck(cudaGraphLaunch(exec, master), "graph launch");
      for (int i : live) s[i]->add_launches(per[i]);
      sipo::ck(cudaStreamSynchronize(master), "batch period");
      std::vector<int> still;
      for (int i : live)
        if (s[i]->host_state().done == 0) still.push_back(i);
      if (still.size() != live.size()) {
        drop_graph();
        live.swap(still);
      }
    }
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
  for (int i = 0; i < n; ++i) s[i]->finish_solve(y_outs ? y_outs[i] : nullptr, y_location, &results[i]);
  return SIPO_OK;
  SIPO_CATCH
}

static int check_dtype(sipo_ctx* ctx, int dtype) {
  if (!ctx) sipo::fail(SIPO_ERR_INVALID_ARG, "null context");
  if (dtype != ctx->c.s->compute_dtype())
    sipo::fail(SIPO_ERR_INVALID_ARG, "dtype must match the context's compute type (F32 for F32/BF16 storage, F64 for F64)");
  return 0;
}

int sipo_project(sipo_ctx* ctx, const void* vol, void* sino, int dtype, void* stream) {
  SIPO_TRY
  check_dtype(ctx, dtype);
  if (!vol || !sino) sipo::fail(SIPO_ERR_INVALID_ARG, "null buffer");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->c.s->strm();
  ctx->c.s->project(vol, sino, s);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_backproject(sipo_ctx* ctx, const void* sino, void* vol, int dtype, void* stream) {
  SIPO_TRY
  check_dtype(ctx, dtype);
  if (!vol || !sino) sipo::fail(SIPO_ERR_INVALID_ARG, "null buffer");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->c.s->strm();
  ctx->c.s->backproject(sino, vol, s);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_psf_apply(sipo_ctx* ctx, const void* in, void* out, int dtype, int deriv_axis, void* stream) {
  SIPO_TRY
  check_dtype(ctx, dtype);
  if (!in || !out || deriv_axis > 2) sipo::fail(SIPO_ERR_INVALID_ARG, "bad argument");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->c.s->strm();
  ctx->c.s->psf_apply(in, out, deriv_axis < 0 ? -1 : deriv_axis, s);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_psf_grad(sipo_ctx* ctx, const void* sino, const void* vol, int dtype, double* grad, void* stream) {
  SIPO_TRY
  check_dtype(ctx, dtype);
  if (!sino || !vol || !grad) sipo::fail(SIPO_ERR_INVALID_ARG, "null buffer");
  cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : ctx->c.s->strm();
  ctx->c.s->psf_grad(sino, vol, grad, s);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_set_psf_sigma(sipo_ctx* ctx, const double sigma[3]) {
  SIPO_TRY
  if (!ctx || !sigma) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  ctx->c.s->set_sigma(sigma);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_get_array(sipo_ctx* ctx, int which, void* out, int location) {
  SIPO_TRY
  if (!ctx || !out) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  ctx->c.s->get_array(which, out, location);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_profile(sipo_ctx* ctx, int iters, double* phase_ms, int n_phases) {
  SIPO_TRY
  if (!ctx || !phase_ms || iters < 0) sipo::fail(SIPO_ERR_INVALID_ARG, "bad argument");
  ctx->c.s->profile(iters, phase_ms, n_phases);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_get_trace(sipo_ctx* ctx, double* out, int max_entries) {
  SIPO_TRY
  if (!ctx || (!out && max_entries > 0)) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  return ctx->c.s->get_trace(out, max_entries);
  SIPO_CATCH
}

int sipo_set_tolerances(sipo_ctx* ctx, const sipo_tolerances* tol) {
  SIPO_TRY
  if (!ctx || !tol) sipo::fail(SIPO_ERR_INVALID_ARG, "null argument");
  ctx->c.s->set_tolerances(tol);
  return SIPO_OK;
  SIPO_CATCH
}

int sipo_destroy(sipo_ctx* ctx) {
  delete ctx;
  return SIPO_OK;
}

}  // extern "C"
