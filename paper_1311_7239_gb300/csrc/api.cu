// C-ABI layer of liblbm.so (declared in include/lbm.h): context lifetime, argument checks,
// host/device pointer handling and kernel dispatch.  No entry point throws; every failure is a
// negative status with a message in lbm_last_error().
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <stdlib.h>

#include <atomic>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local char g_msg[512] = "";

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBM_CUDA(call, what)                 \
  do {                                       \
    cudaError_t e_ = (call);                 \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

}  // namespace

namespace lbm {
// Records msg as the calling thread's last error and returns code (for entry points defined in
// other translation units).
int record_error(int code, const char* msg) { return fail(code, "%s", msg); }

// Kernel parameters of one lattice from its configuration (pointers left null).
void params_from_config(const lbm_config& k, int prec, int pitch, int64_t plane, StepParams& P) {
  memset(&P, 0, sizeof(P));
  P.nx = (int)k.nx;
  P.ny = (int)k.ny;
  P.pitch = pitch;
  P.plane = plane;
  P.bc_x = (int)k.bc_x;
  P.bc_y = (int)k.bc_y;
  P.forch = k.forchheimer ? 1 : 0;
  P.rho0 = (float)k.rho0;
  P.inv_rho0 = (float)(1.0 / k.rho0);
  P.nu = (float)k.nu;
  P.s_e = (float)k.s_e;
  P.s_q = (float)k.s_q;
  const double tau_v = 3.0 * k.J * k.nu + 0.5;  // Eq. 21: J nu = c_s^2 (tau_v - 1/2)
  P.s_v = (float)(1.0 / tau_v);
  P.ax = (float)k.ax;
  P.ay = (float)k.ay;
  P.phi_u = (float)k.phi;
  P.inv_phi_u = (float)(1.0 / k.phi);
  P.c_lin_u = (float)(k.phi * k.nu / k.K);
  P.c_nl_u = k.forchheimer ? (float)(1.75 / sqrt(150.0 * k.phi * k.K)) : 0.0f;
  for (int w = 0; w < 4; ++w) {
    P.Tdir[w] = isnan(k.T_wall[w]) ? 0 : 1;
    P.Tw[w] = isnan(k.T_wall[w]) ? 0.0f : (float)k.T_wall[w];
  }
  P.p_in = (float)k.p_in;
  P.p_out = (float)k.p_out;
  P.p_rest = (float)k.p_rest;
  const double sc = prec == PREC_FP16 ? ldexp(1.0, k.dev_scale_log2) : 1.0;  // only FP16 needs the shift
  P.scale = (float)sc;
  P.inv_scale = (float)(1.0 / sc);
  P.zeta1 = k.thermal ? (float)(1.0 / k.tau_T) : 1.0f;
  P.zeta3 = (float)k.zeta3;
  P.zeta4 = (float)k.zeta4;
  P.inv_sigma = k.sigma > 0 ? (float)(1.0 / k.sigma) : 1.0f;
  P.varpi = 0.0f;  // Appendix B fixes varpi = 0
  P.g_beta = (float)k.g_beta;
  P.T0 = (float)k.T0;
  // constants of the two-cell collision (moments of the stored deviations s d)
  const double rs = k.rho0 * sc, sv = 1.0 / tau_v, hv = 1.0 - 0.5 * sv;
  PairConst& q = P.pc;
  q.inv_rho0s = (float)(1.0 / rs);
  q.nphip = (float)(-2.0 / 3.0 * rs);
  q.nse8 = (float)(-k.s_e / 8.0);
  q.sq6 = (float)(k.s_q / 6.0);
  q.nsq12 = (float)(-k.s_q / 12.0);
  q.r3 = (float)(rs / 3.0);
  q.r12 = (float)(rs / 12.0);
  q.hay = (float)(0.5 * k.ay);
  q.cq = (float)(-0.25 * sv);
  const double c_lin = k.phi * k.nu / k.K, c_nl = k.forchheimer ? 1.75 / sqrt(150.0 * k.phi * k.K) : 0.0;
  const double l0 = 0.5 + 0.25 * c_lin;
  q.u_inv_phi = (float)(1.0 / k.phi);
  q.u_l0 = (float)l0;
  q.u_l0sq = (float)(l0 * l0);
  q.u_l1 = (float)(0.5 * c_nl);
  q.u_nclin = (float)(-c_lin);
  q.u_ncnl = (float)(-c_nl);
  q.u_c2 = (float)(0.1 * (1.0 - 0.5 * k.s_e) * rs / k.phi);
  q.u_nR = (float)(-rs / k.phi);
  q.u_cf7 = (float)(0.5 * hv * rs / k.phi);
  q.u_cf8 = (float)(0.25 * hv * rs / k.phi);
  q.u_hx = (float)(0.5 * k.phi * k.ax);
  q.u_hy = (float)(0.5 * k.phi * k.ay);
  q.k_c2 = (float)(0.1 * (1.0 - 0.5 * k.s_e) * rs);
  q.k_rs = (float)rs;
  q.hax = (float)(0.5 * k.ax);
}

}  // namespace lbm

struct lbm_ctx {
  lbm_config cfg;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int prec = PREC_FP32;
  size_t elem = 4;
  int pitch = 0;
  int64_t plane = 0;
  void* f[2] = {nullptr, nullptr};
  void* g[2] = {nullptr, nullptr};
  int cur = 0;                   // A-B: buffer of the current state; in-place: parity of the next step
  bool inplace = false;          // one buffer (f[0], g[0]) with rows -1..ny and a ghost column; see ip_off
  size_t fbytes = 0, gbytes = 0; // bytes of one flow / temperature population buffer
  float* uprev = nullptr;        // in-place: u before the last step of the last lbm_step call, [2][ny][nx]
  float* edge = nullptr;         // in-place with extrapolated sides: boundary-node states of the coming step
  float* phi = nullptr;
  float* K = nullptr;
  float* sv = nullptr;  // per-cell viscous rate (heterogeneous mode), when a viscosity-ratio field is set
  std::vector<void*> ws;       // adjoint workspace, kept between lbm_adjoint calls (slots, see lbm_adjoint)
  std::vector<size_t> ws_bytes;
  bool het = false;
  unsigned int* err = nullptr;   // device error word
  float* walls = nullptr;        // wall velocities [4][2] read by the kernels
  float* probe = nullptr;        // 4-float read-out slot of lbm_probe
  double* red = nullptr;         // reduction scratch: 2 * kResidualMaxBlocks partials + 2 results
  float* stage = nullptr;        // staging for host inputs/outputs
  size_t stage_bytes = 0;
  uint64_t bytes = 0;
  int64_t steps = 0;
  int64_t history = 0;           // steps since the last initialisation or import
  StepParams base;
  // parameters of the last lbm_init_equilibrium (the initial state the adjoint differentiates)
  double init_p0 = 1.0, init_ux = 0.0, init_uy = 0.0;
  int init_phip = 0;
  // CUDA graphs of kGraphSteps steps starting from buffer 0 or 1 (captured on first use)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
  // adjoint reverse sweep: the adjoint steps on a high-priority stream, the recomputation of the
  // next segment's states on a low-priority one (created on first use)
  cudaStream_t adj_hi = nullptr, adj_lo = nullptr;
  cudaEvent_t adj_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // start, ready[2], freed[2], done
};

namespace {

constexpr int kGraphSteps = 32;  // steps per captured graph (even: a replay ends on the buffer it began on)

bool thermal_of(const lbm_ctx* c) { return c->cfg.thermal != 0; }

// Allocation fault injection for tests: LBM_FAULT_ALLOC=k makes the k-th device allocation of
// the process (counting from 1) fail as if the device were out of memory.
std::atomic<long> g_alloc_count{0};

bool inject_alloc_fault() {
  static const long k = [] {
    const char* v = getenv("LBM_FAULT_ALLOC");
    return v ? atol(v) : 0L;
  }();
  return k > 0 && g_alloc_count.fetch_add(1) + 1 == k;
}

int dev_alloc(lbm_ctx* c, void** p, size_t bytes, const char* what) {
  if (inject_alloc_fault()) {
    *p = nullptr;
    return fail(LBM_ENOMEM, "%s: injected allocation failure (LBM_FAULT_ALLOC)", what);
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  c->bytes += bytes;
  return LBM_OK;
}

// 0: host (or unregistered) memory, 1: device memory of this context's GPU, -1: another GPU
int pointer_kind(const lbm_ctx* c, const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == c->device ? 1 : -1;
  return 0;
}

// Device address of page-locked host memory mapped into the device's address space (pinned memory
// under unified addressing), else nullptr: kernels may write there directly.
float* mapped_host(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<float*>(a.devicePointer) : nullptr;
}

int ensure_stage(lbm_ctx* c, size_t bytes) {
  if (c->stage_bytes >= bytes) return LBM_OK;
  if (c->stage) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->stage);
    c->bytes -= c->stage_bytes;
    c->stage = nullptr;
    c->stage_bytes = 0;
  }
  int rc = dev_alloc(c, reinterpret_cast<void**>(&c->stage), bytes, "cudaMalloc(staging)");
  if (rc == LBM_OK) c->stage_bytes = bytes;
  return rc;
}

// Resolve an input array of n floats to a device pointer (copying host data to the staging
// area at float offset `slot`).
int input_ptr(lbm_ctx* c, const float* user, size_t n, size_t slot, const float** out) {
  *out = nullptr;
  if (!user) return LBM_OK;
  const int kind = pointer_kind(c, user);
  if (kind < 0) return fail(LBM_EINVAL, "input pointer %p is memory of another GPU", (const void*)user);
  if (kind == 1) {
    *out = user;
    return LBM_OK;
  }
  LBM_CUDA(cudaMemcpyAsync(c->stage + slot, user, n * sizeof(float), cudaMemcpyHostToDevice, c->stream), "copy of host input");
  *out = c->stage + slot;
  return LBM_OK;
}

struct OutArg {
  float* user;
  float* dev;
  size_t n;
  bool host;
};

int output_ptr(lbm_ctx* c, float* user, size_t n, size_t slot, OutArg* o) {
  o->user = user;
  o->dev = nullptr;
  o->n = n;
  o->host = false;
  if (!user) return LBM_OK;
  const int kind = pointer_kind(c, user);
  if (kind < 0) return fail(LBM_EINVAL, "output pointer %p is memory of another GPU", (void*)user);
  if (kind == 1) {
    o->dev = user;
    return LBM_OK;
  }
  o->dev = c->stage + slot;
  o->host = true;
  return LBM_OK;
}

int finish_outputs(lbm_ctx* c, OutArg* outs, int n) {
  bool any = false;
  for (int i = 0; i < n; ++i) {
    if (outs[i].user && outs[i].host) {
      LBM_CUDA(cudaMemcpyAsync(outs[i].user, outs[i].dev, outs[i].n * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
               "copy of output to host");
      any = true;
    }
  }
  if (any) LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  return LBM_OK;
}

bool any_host(const lbm_ctx* c, const void* const* ptrs, int n) {
  for (int i = 0; i < n; ++i)
    if (ptrs[i] && pointer_kind(c, ptrs[i]) == 0) return true;
  return false;
}

// row 0 of an in-place buffer (row -1 is the first row of the allocation)
void* ip_row0(const lbm_ctx* c, void* buf) { return buf ? static_cast<char*>(buf) + (size_t)c->pitch * c->elem : nullptr; }

StepParams params_for(const lbm_ctx* c, bool forward_dst = true) {
  StepParams P = c->base;
  if (c->inplace) {
    P.src = P.dst = ip_row0(c, c->f[0]);
    P.gsrc = P.gdst = ip_row0(c, c->g[0]);
    P.parity = c->cur;
  } else {
    P.src = c->f[c->cur];
    P.dst = c->f[c->cur ^ 1];
    P.gsrc = c->g[c->cur];
    P.gdst = c->g[c->cur ^ 1];
  }
  P.phi = c->het ? c->phi : nullptr;
  P.K = c->het ? c->K : nullptr;
  P.sv = c->het ? c->sv : nullptr;
  P.edge = c->inplace ? c->edge : nullptr;
  (void)forward_dst;
  return P;
}

int check_error_word(lbm_ctx* c) {
  unsigned int h = 0;
  LBM_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "read of error word");
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  if (h & 4u) return fail(LBM_ECUDA, "a kernel index left its buffer (debug build check)");
  if (h & 1u) return fail(LBM_EUNSTABLE, "a step produced a non-finite velocity (after %lld steps)", (long long)c->steps);
  return LBM_OK;
}

int validate(const lbm_config* c) {
  return lbm::validate_config(c);
}

}  // namespace

namespace lbm {
int validate_config(const lbm_config* c) {
  if (c->abi_version != LBM_ABI_VERSION) return fail(LBM_EABI, "abi_version %u, library %u", c->abi_version, LBM_ABI_VERSION);
  if (c->nx < 2 || c->ny < 2 || c->nx > 65535 || c->ny > 65535) return fail(LBM_EINVAL, "nx, ny must be in [2, 65535]");
  if (c->precision > LBM_BF16_DEV) return fail(LBM_EINVAL, "unknown precision %u", c->precision);
  if (c->bc_x > LBM_NEE || c->bc_y > LBM_NEE || c->bc_y == LBM_PRESSURE) return fail(LBM_EINVAL, "unknown boundary kind");
  const bool nee = c->bc_x == LBM_NEE || c->bc_y == LBM_NEE;
  if (nee && (c->nx < 3 || c->ny < 3)) return fail(LBM_EINVAL, "extrapolated wall nodes need nx, ny >= 3");
  if (c->bc_x == LBM_PRESSURE && c->nx < 3) return fail(LBM_EINVAL, "pressure columns need nx >= 3");
  if (!(c->nu > 0) || !(c->J > 0) || !(c->rho0 > 0)) return fail(LBM_EINVAL, "nu, J, rho0 must be positive");
  if (!(c->s_e > 0 && c->s_e < 2) || !(c->s_q > 0 && c->s_q < 2)) return fail(LBM_EINVAL, "s_e, s_q must be in (0, 2)");
  if (!(c->phi > 0 && c->phi <= 1) || !(c->K > 0)) return fail(LBM_EINVAL, "uniform phi must be in (0, 1], K > 0");
  if (!isfinite(c->ax) || !isfinite(c->ay) || !isfinite(c->p_rest)) return fail(LBM_EINVAL, "non-finite a or p_rest");
  if (c->dev_scale_log2 < -30 || c->dev_scale_log2 > 30) return fail(LBM_EINVAL, "dev_scale_log2 out of [-30, 30]");
  if (c->streaming > LBM_STREAM_INPLACE) return fail(LBM_EINVAL, "unknown streaming mode %u", c->streaming);
  if (c->options & ~LBM_OPT_NO_RESIDUAL_RECORD) return fail(LBM_EINVAL, "unknown option bits %#x", c->options);
  if (c->thermal) {
    if (!(c->tau_T > 0.5) || !(c->sigma > 0)) return fail(LBM_EINVAL, "tau_T must exceed 1/2 and sigma be positive");
    if (!(c->zeta3 > 0 && c->zeta3 < 2) || !(c->zeta4 > 0 && c->zeta4 < 2)) return fail(LBM_EINVAL, "zeta3, zeta4 in (0, 2)");
  }
  return LBM_OK;
}
}  // namespace lbm

namespace {

void fill_base(lbm_ctx* c) {
  params_from_config(c->cfg, c->prec, c->pitch, c->plane, c->base);
  c->base.uw = c->walls;
  c->base.err = c->err;
  c->base.inplace = c->inplace ? 1 : 0;
}

void drop_graphs(lbm_ctx* c) {
  for (int b = 0; b < 2; ++b) {
    if (c->graph[b]) cudaGraphExecDestroy(c->graph[b]);
    c->graph[b] = nullptr;
  }
}

void release(lbm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  if (c->adj_hi) cudaStreamDestroy(c->adj_hi);
  if (c->adj_lo) cudaStreamDestroy(c->adj_lo);
  for (cudaEvent_t e : c->adj_ev)
    if (e) cudaEventDestroy(e);
  for (int b = 0; b < 2; ++b) {
    cudaFree(c->f[b]);
    cudaFree(c->g[b]);
  }
  cudaFree(c->phi);
  cudaFree(c->K);
  cudaFree(c->sv);
  cudaFree(c->uprev);
  cudaFree(c->edge);
  cudaFree(c->err);
  cudaFree(c->walls);
  cudaFree(c->probe);
  cudaFree(c->red);
  cudaFree(c->stage);
  for (void* p : c->ws) cudaFree(p);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

}  // namespace

extern "C" {

void lbm_config_defaults(lbm_config* cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->abi_version = LBM_ABI_VERSION;
  cfg->nx = cfg->ny = 64;
  cfg->precision = LBM_FP32;
  cfg->bc_x = LBM_PERIODIC;
  cfg->bc_y = LBM_WALL;
  cfg->forchheimer = 1;
  cfg->nu = 0.1;
  cfg->J = 1.0;
  cfg->rho0 = 1.0;
  cfg->s_e = 1.1;
  cfg->s_q = 1.2;
  cfg->phi = 1.0;
  cfg->K = 1e30;
  cfg->p_in = cfg->p_out = 1.0;
  cfg->p_rest = 1.0;
  cfg->dev_scale_log2 = 10;
  cfg->tau_T = 1.0;
  cfg->zeta3 = cfg->zeta4 = 1.1;
  cfg->sigma = 1.0;
  for (int w = 0; w < 4; ++w) cfg->T_wall[w] = NAN;
}

uint32_t lbm_config_size(void) { return (uint32_t)sizeof(lbm_config); }

int lbm_create(const lbm_config* cfg, lbm_ctx** out) {
  if (!cfg || !out) return fail(LBM_EINVAL, "null argument");
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return fail(LBM_ENOMEM, "host allocation of the context");
  c->cfg = *cfg;
  cudaError_t e = cudaGetDevice(&c->device);
  if (e != cudaSuccess) {
    delete c;
    return cuda_fail(e, "cudaGetDevice");
  }
  c->prec = (int)cfg->precision;
  c->elem = c->prec == PREC_FP32 ? 4 : 2;
  // in-place: ghost rows below and above the lattice (rows of the planes) and a ghost column right
  // of it (q columns of ny + 2 slots after the last plane)
  c->inplace = cfg->streaming == LBM_STREAM_INPLACE;
  c->pitch = (int)((cfg->nx + 127) / 128 * 128);
  c->plane = (int64_t)c->pitch * (cfg->ny + (c->inplace ? 2 : 0));
  const int nbuf = c->inplace ? 1 : 2;
  const int64_t ghost_col = c->inplace ? (int64_t)cfg->ny + 2 : 0;
  c->fbytes = 8 * (size_t)(c->plane + ghost_col) * c->elem;
  c->gbytes = 5 * (size_t)(c->plane + ghost_col) * c->elem;
  if (c->inplace && 8 * (uint64_t)(c->plane + ghost_col) > (1ull << 32)) {  // the in-place step indexes with 32-bit offsets
    delete c;
    return fail(LBM_EINVAL, "in-place streaming needs 8 ((ny + 2) pitch + ny + 2) <= 2^32 elements (pitch = nx rounded up to 128)");
  }
  if (cfg->stream) {
    c->stream = static_cast<cudaStream_t>(cfg->stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete c;
      return cuda_fail(e, "cudaStreamCreate");
    }
    c->own_stream = true;
  }
  const size_t fbytes = c->fbytes;
  const size_t gbytes = c->gbytes;
  for (int b = 0; b < nbuf && rc == LBM_OK; ++b) {
    rc = dev_alloc(c, &c->f[b], fbytes, "cudaMalloc(populations)");
    if (rc == LBM_OK && cfg->thermal) rc = dev_alloc(c, &c->g[b], gbytes, "cudaMalloc(temperature populations)");
  }
  if (rc == LBM_OK && c->inplace && !(cfg->options & LBM_OPT_NO_RESIDUAL_RECORD))
    rc = dev_alloc(c, reinterpret_cast<void**>(&c->uprev), 2 * (size_t)cfg->nx * cfg->ny * sizeof(float), "cudaMalloc(previous velocity)");
  if (rc == LBM_OK && c->inplace && (cfg->bc_x == LBM_PRESSURE || cfg->bc_x == LBM_NEE || cfg->bc_y == LBM_NEE))
    rc = dev_alloc(c, reinterpret_cast<void**>(&c->edge), (cfg->thermal ? 13 : 8) * 2 * ((size_t)cfg->nx + cfg->ny) * sizeof(float),
                   "cudaMalloc(boundary-node states)");
  if (rc == LBM_OK) rc = dev_alloc(c, reinterpret_cast<void**>(&c->err), sizeof(unsigned int), "cudaMalloc(error word)");
  if (rc == LBM_OK)
    rc = dev_alloc(c, reinterpret_cast<void**>(&c->red), (2 * kResidualMaxBlocks + 2) * sizeof(double), "cudaMalloc(reduction)");
  if (rc == LBM_OK) rc = dev_alloc(c, reinterpret_cast<void**>(&c->walls), 8 * sizeof(float), "cudaMalloc(walls)");
  if (rc == LBM_OK) rc = dev_alloc(c, reinterpret_cast<void**>(&c->probe), 4 * sizeof(float), "cudaMalloc(probe)");
  if (rc == LBM_OK) {
    float w[8];
    for (int i = 0; i < 8; ++i) w[i] = (float)cfg->u_wall[i / 2][i % 2];
    e = cudaMemcpy(c->walls, w, sizeof(w), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy of wall velocities");
  }
  if (rc == LBM_OK) {
    e = cudaMemsetAsync(c->err, 0, sizeof(unsigned int), c->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset");
  }
  if (rc == LBM_OK) {
    for (int b = 0; b < nbuf && rc == LBM_OK; ++b) {
      e = cudaMemsetAsync(c->f[b], 0, fbytes, c->stream);
      if (e == cudaSuccess && c->g[b]) e = cudaMemsetAsync(c->g[b], 0, gbytes, c->stream);
      if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemset");
    }
  }
  if (rc != LBM_OK) {
    release(c);
    return rc;
  }
  fill_base(c);
  rc = lbm_init_equilibrium(c, 1.0, 0.0, 0.0, 0);
  if (rc == LBM_OK && cfg->thermal) rc = lbm_init_temperature(c, cfg->T0);
  if (rc != LBM_OK) {
    release(c);
    return rc;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* ctx) { release(ctx); }

static int set_medium(lbm_ctx* c, const float* eps, const float* K, int log_k) {
  if (!c) return fail(LBM_EINVAL, "null context");
  drop_graphs(c);  // captured steps bake in the medium mode
  if (!eps && !K && !c->sv) {
    c->het = false;
    return LBM_OK;
  }
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  const size_t fields = (size_t)c->plane * sizeof(float);
  int rc = LBM_OK;
  if (!c->phi) rc = dev_alloc(c, reinterpret_cast<void**>(&c->phi), fields, "cudaMalloc(porosity)");
  if (rc == LBM_OK && !c->K) rc = dev_alloc(c, reinterpret_cast<void**>(&c->K), fields, "cudaMalloc(permeability)");
  if (rc) return rc;
  const void* ptrs[2] = {eps, K};
  if (any_host(c, ptrs, 2) && (rc = ensure_stage(c, 2 * n * sizeof(float)))) return rc;
  const float *de = nullptr, *dk = nullptr;
  if ((rc = input_ptr(c, eps, n, 0, &de)) || (rc = input_ptr(c, K, n, n, &dk))) return rc;
  LBM_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned int), c->stream), "cudaMemset");
  LBM_CUDA(launch_medium(de, dk, (float)c->cfg.phi, (float)c->cfg.K, (int)c->cfg.nx, (int)c->cfg.ny, c->pitch, c->phi, c->K,
                         c->err, log_k, c->stream),
           "medium kernel");
  unsigned int h = 0;
  LBM_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "read of error word");
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  if (h & 2u) {
    LBM_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned int), c->stream), "cudaMemset");
    return fail(LBM_EINVAL, "medium out of range: need 0 < eps <= 1 and 0 < K < 3e38");
  }
  c->het = true;
  return LBM_OK;
}

int lbm_set_medium(lbm_ctx* c, const float* eps, const float* K) { return set_medium(c, eps, K, 0); }

int lbm_set_viscosity_ratio(lbm_ctx* c, const float* J) {
  if (!c) return fail(LBM_EINVAL, "null context");
  drop_graphs(c);
  if (!J) {
    cudaStreamSynchronize(c->stream);
    if (c->sv) {
      cudaFree(c->sv);
      c->bytes -= (uint64_t)c->plane * sizeof(float);
      c->sv = nullptr;
    }
    return LBM_OK;
  }
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  int rc = LBM_OK;
  if (!c->sv && (rc = dev_alloc(c, reinterpret_cast<void**>(&c->sv), (size_t)c->plane * sizeof(float), "cudaMalloc(viscous rate)")))
    return rc;
  if (!c->het) {  // per-cell rates need the heterogeneous kernels: materialise the uniform medium
    if ((rc = set_medium(c, nullptr, nullptr, 0)) && rc != LBM_OK) return rc;
    if (!c->het) {
      const size_t fields = (size_t)c->plane * sizeof(float);
      if (!c->phi && (rc = dev_alloc(c, reinterpret_cast<void**>(&c->phi), fields, "cudaMalloc(porosity)"))) return rc;
      if (!c->K && (rc = dev_alloc(c, reinterpret_cast<void**>(&c->K), fields, "cudaMalloc(permeability)"))) return rc;
      LBM_CUDA(launch_medium(nullptr, nullptr, (float)c->cfg.phi, (float)c->cfg.K, (int)c->cfg.nx, (int)c->cfg.ny, c->pitch, c->phi, c->K,
                             c->err, 0, c->stream),
               "medium kernel");
      c->het = true;
    }
  }
  const void* ptrs[1] = {J};
  if (any_host(c, ptrs, 1) && (rc = ensure_stage(c, n * sizeof(float)))) return rc;
  const float* dJ = nullptr;
  if ((rc = input_ptr(c, J, n, 0, &dJ))) return rc;
  LBM_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned int), c->stream), "cudaMemset");
  LBM_CUDA(launch_viscous_rate(dJ, (int)c->cfg.nx, (int)c->cfg.ny, c->pitch, (float)c->cfg.nu, c->sv, c->err, c->stream),
           "viscous-rate kernel");
  unsigned int h = 0;
  LBM_CUDA(cudaMemcpyAsync(&h, c->err, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "read of error word");
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  if (h & 2u) {
    LBM_CUDA(cudaMemsetAsync(c->err, 0, sizeof(unsigned int), c->stream), "cudaMemset");
    return fail(LBM_EINVAL, "viscosity ratio out of range: need J > 0");
  }
  return LBM_OK;
}

int lbm_set_medium_log(lbm_ctx* c, const float* eps, const float* logK) { return set_medium(c, eps, logK, 1); }

int lbm_init_equilibrium(lbm_ctx* c, double p0, double ux0, double uy0, int phi_p_uniform) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!isfinite(p0) || !isfinite(ux0) || !isfinite(uy0)) return fail(LBM_EINVAL, "non-finite initial state");
  StepParams P = params_for(c);
  if (c->inplace) {
    LBM_CUDA(launch_put_inplace(P, c->prec, c->het, nullptr, nullptr, true, false, (float)p0, (float)ux0, (float)uy0,
                                phi_p_uniform ? 1 : 0, 0.0f, c->stream),
             "init kernel");
  } else {
    P.dst = c->f[c->cur];
    LBM_CUDA(launch_init(P, c->prec, c->het, thermal_of(c), (float)p0, (float)ux0, (float)uy0, phi_p_uniform ? 1 : 0, 0.0f, true,
                         false, c->stream),
             "init kernel");
  }
  c->steps = 0;
  c->history = 0;
  c->init_p0 = p0;
  c->init_ux = ux0;
  c->init_uy = uy0;
  c->init_phip = phi_p_uniform ? 1 : 0;
  return LBM_OK;
}

int lbm_init_temperature(lbm_ctx* c, double T_init) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (!thermal_of(c)) return fail(LBM_ESTATE, "context has no temperature field");
  if (!isfinite(T_init)) return fail(LBM_EINVAL, "non-finite temperature");
  StepParams P = params_for(c);
  if (c->inplace) {
    LBM_CUDA(launch_put_inplace(P, c->prec, c->het, nullptr, nullptr, false, true, 0.0f, 0.0f, 0.0f, 0, (float)T_init, c->stream),
             "init kernel");
  } else {
    P.gdst = c->g[c->cur];
    LBM_CUDA(launch_init(P, c->prec, c->het, true, 0.0f, 0.0f, 0.0f, 0, (float)T_init, false, true, c->stream), "init kernel");
  }
  c->steps = 0;
  c->history = 0;
  return LBM_OK;
}

namespace {

StepParams params_at(const lbm_ctx* c, int cur) {
  StepParams P = params_for(c);
  if (c->inplace) {
    P.parity = cur;
  } else {
    P.src = c->f[cur];
    P.dst = c->f[cur ^ 1];
    P.gsrc = c->g[cur];
    P.gdst = c->g[cur ^ 1];
  }
  return P;
}

// one step from buffer (A-B) or parity (in-place) `cur`
cudaError_t launch_step_at(const lbm_ctx* c, int cur, cudaStream_t s) {
  const StepParams P = params_at(c, cur);
  return c->inplace ? launch_step_inplace(P, c->prec, c->het, thermal_of(c), s) : launch_step(P, c->prec, c->het, thermal_of(c), s);
}

// Instantiate the graph of kGraphSteps steps that starts from buffer `cur`.
int capture_graph(lbm_ctx* c, int cur) {
  if (!c->capture_stream) LBM_CUDA(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  LBM_CUDA(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  cudaError_t launch_err = cudaSuccess;
  for (int k = 0; k < kGraphSteps && launch_err == cudaSuccess; ++k)
    launch_err = launch_step_at(c, cur ^ (k & 1), c->capture_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
  if (launch_err != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(launch_err != cudaSuccess ? launch_err : e, "capture of the step graph");
  }
  e = cudaGraphInstantiate(&c->graph[cur], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->graph[cur] = nullptr;
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  return LBM_OK;
}

}  // namespace

namespace {

int run_steps(lbm_ctx* c, int n) {
  while (n >= kGraphSteps) {  // replay a captured graph of kGraphSteps steps
    if (!c->graph[c->cur]) {
      int rc = capture_graph(c, c->cur);
      if (rc) return rc;
    }
    LBM_CUDA(cudaGraphLaunch(c->graph[c->cur], c->stream), "cudaGraphLaunch");
    c->steps += kGraphSteps;
    c->history += kGraphSteps;
    n -= kGraphSteps;
  }
  for (int k = 0; k < n; ++k) {
    LBM_CUDA(launch_step_at(c, c->cur, c->stream), "step kernel");
    c->cur ^= 1;
    ++c->steps;
    ++c->history;
  }
  return LBM_OK;
}

}  // namespace

int lbm_step(lbm_ctx* c, int n) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (n < 0) return fail(LBM_EINVAL, "negative step count");
  if (!c->uprev || n == 0) return run_steps(c, n);
  // in-place: the last step records the velocity of its collisions, u(t-1) of the residual once it
  // is done (the state it came from is overwritten)
  int rc = run_steps(c, n - 1);
  if (rc) return rc;
  StepParams P = params_at(c, c->cur);
  P.urec = c->uprev;
  LBM_CUDA(launch_step_inplace(P, c->prec, c->het, thermal_of(c), c->stream), "step kernel");
  c->cur ^= 1;
  ++c->steps;
  ++c->history;
  return LBM_OK;
}

int lbm_set_walls(lbm_ctx* c, const float* u_wall) {
  if (!c || !u_wall) return fail(LBM_EINVAL, "null argument");
  const int kind = pointer_kind(c, u_wall);
  if (kind < 0) return fail(LBM_EINVAL, "wall velocities in memory of another GPU");
  // page-locked host memory: read by a one-warp kernel (a launch on the stream, no copy-engine
  // hand-over between the steps); other memory: a copy
  const float* mapped = kind ? nullptr : mapped_host(u_wall);
  if (mapped)
    LBM_CUDA(launch_copy_small(c->walls, mapped, 8, c->stream), "copy of wall velocities");
  else
    LBM_CUDA(cudaMemcpyAsync(c->walls, u_wall, 8 * sizeof(float), kind ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream),
             "copy of wall velocities");
  for (int i = 0; i < 8; ++i)
    if (kind == 0) c->cfg.u_wall[i / 2][i % 2] = u_wall[i];
  return LBM_OK;
}

int lbm_probe(lbm_ctx* c, int x, int y, float* out) {
  if (!c || !out) return fail(LBM_EINVAL, "null argument");
  if (x < 0 || y < 0 || x >= (int)c->cfg.nx || y >= (int)c->cfg.ny) return fail(LBM_EINVAL, "probe cell outside the lattice");
  const int kind = pointer_kind(c, out);
  if (kind < 0) return fail(LBM_EINVAL, "probe output in memory of another GPU");
  StepParams P = params_for(c);
  float* mapped = kind ? nullptr : mapped_host(out);  // pinned host memory: written by the kernel
  LBM_CUDA(launch_probe(P, c->prec, c->het, thermal_of(c), x, y, kind ? out : (mapped ? mapped : c->probe), c->stream), "probe kernel");
  if (kind == 0) {
    if (!mapped) LBM_CUDA(cudaMemcpyAsync(out, c->probe, 4 * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy of probe");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  }
  return LBM_OK;
}

int lbm_probe_async(lbm_ctx* c, int x, int y, float* out) {
  if (!c || !out) return fail(LBM_EINVAL, "null argument");
  if (x < 0 || y < 0 || x >= (int)c->cfg.nx || y >= (int)c->cfg.ny) return fail(LBM_EINVAL, "probe cell outside the lattice");
  const int kind = pointer_kind(c, out);
  if (kind < 0) return fail(LBM_EINVAL, "probe output in memory of another GPU");
  StepParams P = params_for(c);
  // pinned host memory: the kernel writes it directly; pageable: through the device slot and a copy
  // (the next probe kernel on the stream runs after this copy has read the slot)
  float* mapped = kind ? nullptr : mapped_host(out);
  LBM_CUDA(launch_probe(P, c->prec, c->het, thermal_of(c), x, y, kind ? out : (mapped ? mapped : c->probe), c->stream), "probe kernel");
  if (kind == 0 && !mapped)
    LBM_CUDA(cudaMemcpyAsync(out, c->probe, 4 * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy of probe");
  return LBM_OK;
}

int lbm_macros(lbm_ctx* c, float* p, float* ux, float* uy, float* T) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (T && !thermal_of(c)) return fail(LBM_ESTATE, "context has no temperature field");
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  const void* ptrs[4] = {p, ux, uy, T};
  int rc;
  if (any_host(c, ptrs, 4) && (rc = ensure_stage(c, 4 * n * sizeof(float)))) return rc;
  OutArg o[4];
  float* users[4] = {p, ux, uy, T};
  for (int i = 0; i < 4; ++i)
    if ((rc = output_ptr(c, users[i], n, i * n, &o[i]))) return rc;
  StepParams P = params_for(c);
  LBM_CUDA(launch_macros(P, c->prec, c->het, thermal_of(c), o[0].dev, o[1].dev, o[2].dev, o[3].dev, c->stream), "macros kernel");
  return finish_outputs(c, o, 4);
}

int lbm_get_populations(lbm_ctx* c, float* f, float* g) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (g && !thermal_of(c)) return fail(LBM_ESTATE, "context has no temperature field");
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  const void* ptrs[2] = {f, g};
  int rc;
  if (any_host(c, ptrs, 2) && (rc = ensure_stage(c, 13 * n * sizeof(float)))) return rc;
  OutArg o[2];
  if ((rc = output_ptr(c, f, 8 * n, 0, &o[0])) || (rc = output_ptr(c, g, 5 * n, 8 * n, &o[1]))) return rc;
  StepParams P = params_for(c);
  LBM_CUDA(launch_export(P, c->prec, c->het, thermal_of(c), o[0].dev, o[1].dev, c->stream), "export kernel");
  return finish_outputs(c, o, 2);
}

int lbm_set_populations(lbm_ctx* c, const float* f, const float* g) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (g && !thermal_of(c)) return fail(LBM_ESTATE, "context has no temperature field");
  const size_t n = (size_t)c->cfg.nx * c->cfg.ny;
  const void* ptrs[2] = {f, g};
  int rc;
  if (any_host(c, ptrs, 2) && (rc = ensure_stage(c, 13 * n * sizeof(float)))) return rc;
  const float *df = nullptr, *dg = nullptr;
  if ((rc = input_ptr(c, f, 8 * n, 0, &df)) || (rc = input_ptr(c, g, 5 * n, 8 * n, &dg))) return rc;
  StepParams P = params_for(c);
  if (c->inplace) {
    LBM_CUDA(launch_put_inplace(P, c->prec, c->het, df, dg, df != nullptr, dg != nullptr, 0.0f, 0.0f, 0.0f, 0, 0.0f, c->stream),
             "import kernel");
  } else {
    P.dst = c->f[c->cur];
    P.gdst = c->g[c->cur];
    LBM_CUDA(launch_import(P, c->prec, df, dg, c->stream), "import kernel");
  }
  c->history = 0;
  if (any_host(c, ptrs, 2)) LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  return LBM_OK;
}

int lbm_residual(lbm_ctx* c, double* r) {
  if (!c || !r) return fail(LBM_EINVAL, "null argument");
  if (c->history < 1) return fail(LBM_ESTATE, "the residual needs one step since the last initialisation");
  if (c->inplace && !c->uprev) return fail(LBM_ESTATE, "in-place context created with LBM_OPT_NO_RESIDUAL_RECORD");
  StepParams P = params_for(c);
  const int nb = residual_blocks((int)c->cfg.nx, (int)c->cfg.ny);
  double* out = c->red + 2 * kResidualMaxBlocks;
  if (c->inplace)
    LBM_CUDA(launch_residual(P, c->prec, c->het, thermal_of(c), nullptr, nullptr, c->uprev, c->red, nb, out, c->stream),
             "residual kernels");
  else
    LBM_CUDA(launch_residual(P, c->prec, c->het, thermal_of(c), c->f[c->cur ^ 1], c->g[c->cur ^ 1], nullptr, c->red, nb, out,
                             c->stream),
             "residual kernels");
  double h[2];
  LBM_CUDA(cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "read of residual");
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  *r = h[1] > 0 ? sqrt(h[0] / h[1]) : 0.0;
  return check_error_word(c);
}

int lbm_nusselt(lbm_ctx* c, int side, double* nu) {
  if (!c || !nu) return fail(LBM_EINVAL, "null argument");
  if (!thermal_of(c)) return fail(LBM_ESTATE, "context has no temperature field");
  if (side != LBM_LEFT && side != LBM_RIGHT) return fail(LBM_EINVAL, "side must be LBM_LEFT or LBM_RIGHT");
  if ((c->cfg.bc_x != LBM_WALL && c->cfg.bc_x != LBM_NEE) || isnan(c->cfg.T_wall[LBM_LEFT]) || isnan(c->cfg.T_wall[LBM_RIGHT]))
    return fail(LBM_ESTATE, "the Nusselt number needs isothermal left and right walls");
  const double dT = c->cfg.T_wall[LBM_LEFT] - c->cfg.T_wall[LBM_RIGHT];
  if (dT == 0) return fail(LBM_EINVAL, "equal wall temperatures");
  StepParams P = params_for(c);
  double* out = c->red + 2 * kResidualMaxBlocks;
  LBM_CUDA(launch_nusselt(P, c->prec, side, out, c->stream), "nusselt kernel");
  double s = 0;
  LBM_CUDA(cudaMemcpyAsync(&s, out, sizeof(s), cudaMemcpyDeviceToHost, c->stream), "read of Nusselt sum");
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  const int rows = (int)c->cfg.ny - (c->cfg.bc_x == LBM_NEE && c->cfg.bc_y == LBM_NEE ? 2 : 0);
  const double mean = s / (double)rows;
  const double width = c->cfg.bc_x == LBM_NEE ? (double)c->cfg.nx - 1.0 : (double)c->cfg.nx;  // wall-to-wall distance
  *nu = (side == LBM_LEFT ? -1.0 : 1.0) * width / dT * mean;
  return check_error_word(c);
}

namespace {

// Device buffers of one adjoint run, freed on every exit path.
// Slot k of the adjoint workspace, `bytes` long: the buffer kept from an earlier call when its
// size matches, else a new allocation.  Callers synchronise before the workspace changes hands.
void* ws_slot(lbm_ctx* c, size_t k, size_t bytes, int* rc, const char* what) {
  if (c->ws.size() <= k) {
    c->ws.resize(k + 1, nullptr);
    c->ws_bytes.resize(k + 1, 0);
  }
  if (c->ws[k] && c->ws_bytes[k] == bytes) return c->ws[k];
  if (c->ws[k]) {
    cudaFree(c->ws[k]);
    c->bytes -= c->ws_bytes[k];
    c->ws[k] = nullptr;
    c->ws_bytes[k] = 0;
  }
  void* p = nullptr;
  if ((*rc = dev_alloc(c, &p, bytes, what)) != LBM_OK) return nullptr;
  c->ws[k] = p;
  c->ws_bytes[k] = bytes;
  return p;
}

// Frees the workspace slots from `keep` on.
void ws_trim(lbm_ctx* c, size_t keep) {
  for (size_t k = keep; k < c->ws.size(); ++k) {
    if (c->ws[k]) {
      cudaFree(c->ws[k]);
      c->bytes -= c->ws_bytes[k];
    }
  }
  if (c->ws.size() > keep) {
    c->ws.resize(keep);
    c->ws_bytes.resize(keep);
  }
}

int copy_out(lbm_ctx* c, void* user, const void* dev, size_t bytes, bool* waited) {
  if (!user) return LBM_OK;
  const int kind = pointer_kind(c, user);
  if (kind < 0) return fail(LBM_EINVAL, "output in memory of another GPU");
  LBM_CUDA(cudaMemcpyAsync(user, dev, bytes, kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream), "copy of output");
  if (!kind) *waited = true;
  return LBM_OK;
}

// pitched FP64 field [ny][pitch] -> dense caller array [ny][nx]
int copy_out_rows(lbm_ctx* c, double* user, const double* dev, bool* waited) {
  if (!user) return LBM_OK;
  const int kind = pointer_kind(c, user);
  if (kind < 0) return fail(LBM_EINVAL, "output in memory of another GPU");
  LBM_CUDA(cudaMemcpy2DAsync(user, c->cfg.nx * sizeof(double), dev, (size_t)c->pitch * sizeof(double), c->cfg.nx * sizeof(double),
                             c->cfg.ny, kind ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
           "copy of gradient");
  if (!kind) *waited = true;
  return LBM_OK;
}

}  // namespace

int lbm_adjoint(lbm_ctx* c, int T, int loss_kind, const float* target_ux, const float* target_uy, double* grad_logK,
                double* grad_eps, double* loss) {
  if (!c) return fail(LBM_EINVAL, "null context");
  if (T < 1) return fail(LBM_EINVAL, "T must be at least 1");
  if (loss_kind != LBM_LOSS_OUTLET_FLUX && loss_kind != LBM_LOSS_VELOCITY_MISFIT) return fail(LBM_EINVAL, "unknown loss kind");
  if (loss_kind == LBM_LOSS_VELOCITY_MISFIT && (!target_ux || !target_uy)) return fail(LBM_EINVAL, "misfit loss needs a target");
  if (thermal_of(c)) return fail(LBM_ESTATE, "the adjoint covers the isothermal flow step only");
  if ((c->cfg.bc_x == LBM_NEE && c->cfg.nx < 4) || (c->cfg.bc_y == LBM_NEE && c->cfg.ny < 4))
    return fail(LBM_EINVAL, "the adjoint through extrapolated wall nodes needs at least 4 nodes across each such side pair");
  if (c->steps != 0 || c->history != 0)
    return fail(LBM_ESTATE, "lbm_adjoint differentiates from the initial state: call lbm_init_equilibrium first");
  const int64_t n = (int64_t)c->cfg.nx * c->cfg.ny;
  const size_t fbytes = 8 * (size_t)c->plane * c->elem;
  const size_t nubytes = 8 * (size_t)c->plane * sizeof(float);
  int ck = 1;
  while ((int64_t)ck * ck < T) ++ck;  // checkpoint interval ceil(sqrt(T))
  const int nck = (T + ck - 1) / ck;
  // workspace slots (kept between calls): 0-1 adjoint state, 2-3 FP64 gradient totals, 4-5 FP32
  // gradient partial sums, then nck checkpoints and two sets of ck segment states
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  int rc = LBM_OK;
  float* nu[2];
  for (int b = 0; b < 2; ++b)
    if (!(nu[b] = static_cast<float*>(ws_slot(c, b, nubytes, &rc, "cudaMalloc(adjoint state)")))) return rc;
  const size_t gbytes = (size_t)c->plane * sizeof(double);  // pitched [ny][pitch]
  const size_t hbytes = (size_t)c->plane * sizeof(float);
  double* gl = static_cast<double*>(ws_slot(c, 2, gbytes, &rc, "cudaMalloc(gradients)"));
  double* gp = gl ? static_cast<double*>(ws_slot(c, 3, gbytes, &rc, "cudaMalloc(gradients)")) : nullptr;
  float* hl = gp ? static_cast<float*>(ws_slot(c, 4, hbytes, &rc, "cudaMalloc(gradient partial sums)")) : nullptr;
  float* hp = hl ? static_cast<float*>(ws_slot(c, 5, hbytes, &rc, "cudaMalloc(gradient partial sums)")) : nullptr;
  if (!hp) return rc;
  // two sets of segment states: the adjoint steps of one segment read one set while the states of
  // the segment before it are recomputed into the other
  std::vector<void*> ckpt(nck), seg[2] = {std::vector<void*>(ck), std::vector<void*>(ck)};
  for (int k = 0; k < nck; ++k)
    if (!(ckpt[k] = ws_slot(c, 6 + k, fbytes, &rc, "cudaMalloc(checkpoints)"))) return rc;
  for (int h = 0; h < 2; ++h)
    for (int j = 0; j < ck; ++j)
      if (!(seg[h][j] = ws_slot(c, 6 + nck + h * ck + j, fbytes, &rc, "cudaMalloc(segment states)"))) return rc;
  // In-place contexts: the sweep runs on two A-B state buffers of the workspace, from the same
  // initial state and with the same kernels as an A-B context; the final state is then written back
  // into the in-place layout (and the velocity of step T - 1 into the residual's record).
  const bool ip = c->inplace;
  void* ab[2] = {c->f[0], c->f[1]};
  for (int b = 0; ip && b < 2; ++b)
    if (!(ab[b] = ws_slot(c, 6 + nck + 2 * ck + b, fbytes, &rc, "cudaMalloc(A-B states)"))) return rc;
  ws_trim(c, 6 + nck + 2 * ck + (ip ? 2 : 0));
  if (ip && (rc = ensure_stage(c, 10 * n * sizeof(float)))) return rc;  // targets, then the final state
  StepParams B = params_for(c);
  B.inplace = 0;
  B.parity = 0;
  B.edge = nullptr;
  B.urec = nullptr;
  int cur = ip ? 0 : c->cur;
  auto ab_params = [&](int k) {
    StepParams Q = B;
    Q.src = ab[k];
    Q.dst = ab[k ^ 1];
    return Q;
  };
  if (ip)
    LBM_CUDA(launch_init(ab_params(1), c->prec, c->het, false, (float)c->init_p0, (float)c->init_ux, (float)c->init_uy, c->init_phip,
                         0.0f, true, false, c->stream),
             "init kernel");
  if (!c->adj_hi) {
    int least = 0, greatest = 0;
    LBM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest), "cudaDeviceGetStreamPriorityRange");
    LBM_CUDA(cudaStreamCreateWithPriority(&c->adj_hi, cudaStreamNonBlocking, greatest), "cudaStreamCreate");
    LBM_CUDA(cudaStreamCreateWithPriority(&c->adj_lo, cudaStreamNonBlocking, least), "cudaStreamCreate");
    for (cudaEvent_t& e : c->adj_ev) LBM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
  }
  cudaStream_t hi = c->adj_hi, lo = c->adj_lo;
  cudaEvent_t ev_start = c->adj_ev[0], ev_done = c->adj_ev[5];
  cudaEvent_t ready[2] = {c->adj_ev[1], c->adj_ev[2]}, freed[2] = {c->adj_ev[3], c->adj_ev[4]};
  for (int b = 0; b < 2; ++b) LBM_CUDA(cudaMemsetAsync(nu[b], 0, nubytes, c->stream), "cudaMemset");
  const float *tux = nullptr, *tuy = nullptr;
  if (loss_kind == LBM_LOSS_VELOCITY_MISFIT) {
    const void* ptrs[2] = {target_ux, target_uy};
    if (any_host(c, ptrs, 2) && (rc = ensure_stage(c, 2 * n * sizeof(float)))) return rc;
    if ((rc = input_ptr(c, target_ux, n, 0, &tux)) || (rc = input_ptr(c, target_uy, n, n, &tuy))) return rc;
  }
  LBM_CUDA(cudaMemsetAsync(gl, 0, gbytes, c->stream), "cudaMemset");
  LBM_CUDA(cudaMemsetAsync(gp, 0, gbytes, c->stream), "cudaMemset");
  LBM_CUDA(cudaMemsetAsync(hl, 0, hbytes, c->stream), "cudaMemset");
  LBM_CUDA(cudaMemsetAsync(hp, 0, hbytes, c->stream), "cudaMemset");
  const bool pressure = c->cfg.bc_x == LBM_PRESSURE;
  // forward sweep, keeping the buffer before every ck-th step
  for (int t = 0; t < T; ++t) {
    if (t % ck == 0)
      LBM_CUDA(cudaMemcpyAsync(ckpt[t / ck], ab[cur], fbytes, cudaMemcpyDeviceToDevice, c->stream), "checkpoint copy");
    LBM_CUDA(launch_step(ab_params(cur), c->prec, c->het, false, c->stream), "step kernel");
    cur ^= 1;
    ++c->steps;
    ++c->history;
  }
  if (!ip) c->cur = cur;
  StepParams P = ab_params(cur);
  const int nb = residual_blocks((int)c->cfg.nx, (int)c->cfg.ny);
  double* loss_dev = c->red + 2 * kResidualMaxBlocks;
  LBM_CUDA(launch_adj_seed(P, c->prec, c->het, nu[0], hl, hp, loss_kind, tux, tuy, c->red, nb, loss_dev, c->stream), "adjoint seed");
  const bool walls = c->cfg.bc_x == LBM_NEE || c->cfg.bc_y == LBM_NEE;
  // J_N^T of the boundary nodes N = (wall nodes) o (pressure columns): wall nodes first
  if (walls) LBM_CUDA(launch_adj_wall(P, c->prec, c->het, ab[cur], nu[0], hl, hp, c->stream), "adjoint wall nodes");
  if (pressure) LBM_CUDA(launch_adj_nee(P, c->prec, c->het, ab[cur], nu[0], hl, hp, c->stream), "adjoint pressure columns");
  if (ip) {  // the state after step T into the in-place layout; u of step T - 1 into the record
    // (moved as deviations, p_rest = 0 on both sides, so that no rest value is added and taken off
    // again; the boundary nodes' own values, which that changes, are never read: the in-place step
    // and the read-outs extrapolate them from their inner neighbours)
    float* dense = c->stage + 2 * n;
    StepParams E = ab_params(cur), I = params_at(c, c->cur);
    E.p_rest = 0.0f;
    I.p_rest = 0.0f;
    LBM_CUDA(launch_export(E, c->prec, c->het, false, dense, nullptr, c->stream), "export kernel");
    LBM_CUDA(launch_put_inplace(I, c->prec, c->het, dense, nullptr, true, false, 0.0f, 0.0f, 0.0f, 0, 0.0f, c->stream),
             "in-place put kernel");
    if (c->uprev)
      LBM_CUDA(launch_macros(ab_params(cur ^ 1), c->prec, c->het, false, nullptr, c->uprev, c->uprev + n, nullptr, c->stream),
               "record of u(t-1)");
  }
  int cur_nu = 0, unfolded = 1;
  constexpr int kAdjFold = 64;  // at most this many per-step terms in an FP32 partial sum
  // Reverse sweep over the segments, last first.  The states of segment k - 1 are recomputed from
  // its checkpoint on the low-priority stream while the adjoint steps of segment k run on the
  // high-priority one (whose small boundary-transpose launches and tails leave the SMs partly
  // idle); set k & 1 holds segment k's states, and the recomputation into a set waits until the
  // adjoint steps that read it (segment k + 2) are done.
  LBM_CUDA(cudaEventRecord(ev_start, c->stream), "cudaEventRecord");
  LBM_CUDA(cudaStreamWaitEvent(hi, ev_start, 0), "cudaStreamWaitEvent");
  LBM_CUDA(cudaStreamWaitEvent(lo, ev_start, 0), "cudaStreamWaitEvent");
  for (int h = 0; h < 2; ++h) LBM_CUDA(cudaEventRecord(freed[h], hi), "cudaEventRecord");
  auto recompute = [&](int k) -> int {
    const int t0 = k * ck, t1 = (t0 + ck < T) ? t0 + ck : T;
    std::vector<void*>& S = seg[k & 1];
    LBM_CUDA(cudaStreamWaitEvent(lo, freed[k & 1], 0), "cudaStreamWaitEvent");
    LBM_CUDA(cudaMemcpyAsync(S[0], ckpt[k], fbytes, cudaMemcpyDeviceToDevice, lo), "checkpoint restore");
    for (int j = 1; j < t1 - t0; ++j) {
      StepParams F = P;
      F.src = S[j - 1];
      F.dst = S[j];
      LBM_CUDA(launch_step(F, c->prec, c->het, false, lo), "recompute step");
    }
    LBM_CUDA(cudaEventRecord(ready[k & 1], lo), "cudaEventRecord");
    return LBM_OK;
  };
  auto sweep = [&]() -> int {
    int rc2 = recompute(nck - 1);
    if (rc2) return rc2;
    for (int k = nck - 1; k >= 0; --k) {
      const int t0 = k * ck, t1 = (t0 + ck < T) ? t0 + ck : T;
      if (k > 0 && (rc2 = recompute(k - 1))) return rc2;
      LBM_CUDA(cudaStreamWaitEvent(hi, ready[k & 1], 0), "cudaStreamWaitEvent");
      for (int t = t1 - 1; t >= t0; --t) {
        const void* buf = seg[k & 1][t - t0];
        LBM_CUDA(launch_adj_step(P, c->prec, c->het, buf, nu[cur_nu], nu[cur_nu ^ 1], hl, hp, hi), "adjoint step");
        cur_nu ^= 1;
        if (walls) LBM_CUDA(launch_adj_wall(P, c->prec, c->het, buf, nu[cur_nu], hl, hp, hi), "adjoint wall nodes");
        if (pressure) LBM_CUDA(launch_adj_nee(P, c->prec, c->het, buf, nu[cur_nu], hl, hp, hi), "adjoint pressure columns");
        if (++unfolded == kAdjFold) {
          LBM_CUDA(launch_adj_fold(hl, hp, gl, gp, c->plane, hi), "gradient fold");
          unfolded = 0;
        }
      }
      LBM_CUDA(cudaEventRecord(freed[k & 1], hi), "cudaEventRecord");
    }
    return LBM_OK;
  };
  if ((rc = sweep())) {  // nothing of the sweep may still run when the workspace changes hands
    cudaStreamSynchronize(hi);
    cudaStreamSynchronize(lo);
    return rc;
  }
  LBM_CUDA(cudaEventRecord(ev_done, hi), "cudaEventRecord");
  LBM_CUDA(cudaStreamWaitEvent(c->stream, ev_done, 0), "cudaStreamWaitEvent");
  LBM_CUDA(launch_adj_init(P, c->het, nu[cur_nu], hp, (float)c->init_p0, (float)c->init_ux, (float)c->init_uy, c->init_phip, c->stream),
           "adjoint initial state");
  LBM_CUDA(launch_adj_fold(hl, hp, gl, gp, c->plane, c->stream), "gradient fold");
  bool waited = false;
  if ((rc = copy_out_rows(c, grad_logK, gl, &waited)) || (rc = copy_out_rows(c, grad_eps, gp, &waited)) ||
      (rc = copy_out(c, loss, loss_dev, sizeof(double), &waited)))
    return rc;
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");  // the workspace may be reused or freed after return
  return check_error_word(c);
}

int lbm_adjoint_step(lbm_ctx* c, int T, int loss_kind, const float* target_ux, const float* target_uy, double* grad_logK,
                     double* grad_eps, double* loss) {
  return lbm_adjoint(c, T, loss_kind, target_ux, target_uy, grad_logK, grad_eps, loss);
}

int lbm_release_workspace(lbm_ctx* c) {
  if (!c) return fail(LBM_EINVAL, "null context");
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  ws_trim(c, 0);
  return LBM_OK;
}

namespace {

constexpr uint32_t kSaveMagic = 0x4C424D53u;  // "LBMS"
constexpr uint32_t kSaveVersion = 3u;

struct SaveHeader {
  uint32_t magic, version, config_size, precision;
  uint32_t nx, ny, pitch, thermal;
  int32_t cur, het, init_phip, inplace;
  int64_t steps, history;
  double init_p0, init_ux, init_uy;
  uint64_t pop_bytes, therm_bytes, medium_bytes, sv_bytes;
};

int io_fail(FILE* f, const char* what) {
  if (f) fclose(f);
  return fail(LBM_EINVAL, "%s", what);
}

}  // namespace

int lbm_save(lbm_ctx* c, const char* path) {
  if (!c || !path) return fail(LBM_EINVAL, "null argument");
  SaveHeader h;
  memset(&h, 0, sizeof(h));
  h.magic = kSaveMagic;
  h.version = kSaveVersion;
  h.config_size = (uint32_t)sizeof(lbm_config);
  h.precision = (uint32_t)c->prec;
  h.nx = c->cfg.nx;
  h.ny = c->cfg.ny;
  h.pitch = (uint32_t)c->pitch;
  h.thermal = c->cfg.thermal ? 1u : 0u;
  h.cur = c->cur;
  h.het = c->het ? 1 : 0;
  h.init_phip = c->init_phip;
  h.inplace = c->inplace ? (c->uprev ? 1 : 2) : 0;  // 1: with the u(t-1) record
  h.steps = c->steps;
  h.history = c->history;
  h.init_p0 = c->init_p0;
  h.init_ux = c->init_ux;
  h.init_uy = c->init_uy;
  h.pop_bytes = c->fbytes;
  h.therm_bytes = c->cfg.thermal ? c->gbytes : 0;
  h.medium_bytes = c->het ? (uint64_t)c->plane * sizeof(float) : 0;
  h.sv_bytes = (c->het && c->sv) ? (uint64_t)c->plane * sizeof(float) : 0;
  std::vector<char> host(h.pop_bytes > h.medium_bytes ? h.pop_bytes : h.medium_bytes);
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(LBM_EINVAL, "cannot open %s for writing", path);
  lbm_config cfg = c->cfg;
  cfg.stream = nullptr;
  if (fwrite(&h, sizeof(h), 1, f) != 1 || fwrite(&cfg, sizeof(cfg), 1, f) != 1) return io_fail(f, "write failed");
  // both population buffers (the previous one serves the residual; in-place: the one buffer and
  // the recorded u(t-1)), temperature, medium
  for (int b = 0; b < (c->inplace ? 1 : 2); ++b) {
    if (cudaMemcpy(host.data(), c->f[b], h.pop_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return io_fail(f, "device read failed");
    if (fwrite(host.data(), 1, h.pop_bytes, f) != h.pop_bytes) return io_fail(f, "write failed");
    if (h.therm_bytes) {
      if (cudaMemcpy(host.data(), c->g[b], h.therm_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return io_fail(f, "device read failed");
      if (fwrite(host.data(), 1, h.therm_bytes, f) != h.therm_bytes) return io_fail(f, "write failed");
    }
  }
  if (c->uprev) {
    const size_t ub = 2 * (size_t)c->cfg.nx * c->cfg.ny * sizeof(float);
    std::vector<char> u(ub);
    if (cudaMemcpy(u.data(), c->uprev, ub, cudaMemcpyDeviceToHost) != cudaSuccess) return io_fail(f, "device read failed");
    if (fwrite(u.data(), 1, ub, f) != ub) return io_fail(f, "write failed");
  }
  if (h.medium_bytes) {
    float* fields[2] = {c->phi, c->K};
    for (int k = 0; k < 2; ++k) {
      if (cudaMemcpy(host.data(), fields[k], h.medium_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return io_fail(f, "device read failed");
      if (fwrite(host.data(), 1, h.medium_bytes, f) != h.medium_bytes) return io_fail(f, "write failed");
    }
  }
  if (h.sv_bytes) {
    if (cudaMemcpy(host.data(), c->sv, h.sv_bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return io_fail(f, "device read failed");
    if (fwrite(host.data(), 1, h.sv_bytes, f) != h.sv_bytes) return io_fail(f, "write failed");
  }
  if (fclose(f) != 0) return fail(LBM_EINVAL, "close of %s failed", path);
  return LBM_OK;
}

int lbm_load(lbm_ctx* c, const char* path) {
  if (!c || !path) return fail(LBM_EINVAL, "null argument");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(LBM_EINVAL, "cannot open %s", path);
  SaveHeader h;
  lbm_config cfg;
  if (fread(&h, sizeof(h), 1, f) != 1 || h.magic != kSaveMagic) return io_fail(f, "not a liblbm state file");
  if (h.version != kSaveVersion || h.config_size != sizeof(lbm_config)) return io_fail(f, "state file of another format version");
  if (fread(&cfg, sizeof(cfg), 1, f) != 1) return io_fail(f, "truncated state file");
  if (h.nx != c->cfg.nx || h.ny != c->cfg.ny || (int)h.precision != c->prec || (h.thermal != 0) != (c->cfg.thermal != 0) ||
      (int)h.pitch != c->pitch || h.inplace != (c->inplace ? (c->uprev ? 1 : 2) : 0))
    return io_fail(f, "state file does not match the context (size, precision, thermal, streaming or residual record)");
  if (h.pop_bytes != c->fbytes) return io_fail(f, "state file layout mismatch");
  std::vector<char> host(h.pop_bytes > h.medium_bytes ? h.pop_bytes : h.medium_bytes);
  LBM_CUDA(cudaStreamSynchronize(c->stream), "stream synchronize");
  for (int b = 0; b < (c->inplace ? 1 : 2); ++b) {
    if (fread(host.data(), 1, h.pop_bytes, f) != h.pop_bytes) return io_fail(f, "truncated state file");
    if (cudaMemcpy(c->f[b], host.data(), h.pop_bytes, cudaMemcpyHostToDevice) != cudaSuccess) return io_fail(f, "device write failed");
    if (h.therm_bytes) {
      if (fread(host.data(), 1, h.therm_bytes, f) != h.therm_bytes) return io_fail(f, "truncated state file");
      if (cudaMemcpy(c->g[b], host.data(), h.therm_bytes, cudaMemcpyHostToDevice) != cudaSuccess)
        return io_fail(f, "device write failed");
    }
  }
  if (c->uprev) {
    const size_t ub = 2 * (size_t)c->cfg.nx * c->cfg.ny * sizeof(float);
    std::vector<char> u(ub);
    if (fread(u.data(), 1, ub, f) != ub) return io_fail(f, "truncated state file");
    if (cudaMemcpy(c->uprev, u.data(), ub, cudaMemcpyHostToDevice) != cudaSuccess) return io_fail(f, "device write failed");
  }
  drop_graphs(c);
  if (h.medium_bytes) {
    const size_t fields = (size_t)c->plane * sizeof(float);
    int rc = LBM_OK;
    if (!c->phi) rc = dev_alloc(c, reinterpret_cast<void**>(&c->phi), fields, "cudaMalloc(porosity)");
    if (rc == LBM_OK && !c->K) rc = dev_alloc(c, reinterpret_cast<void**>(&c->K), fields, "cudaMalloc(permeability)");
    if (rc) {
      fclose(f);
      return rc;
    }
    float* dst[2] = {c->phi, c->K};
    for (int k = 0; k < 2; ++k) {
      if (fread(host.data(), 1, h.medium_bytes, f) != h.medium_bytes) return io_fail(f, "truncated state file");
      if (cudaMemcpy(dst[k], host.data(), h.medium_bytes, cudaMemcpyHostToDevice) != cudaSuccess) return io_fail(f, "device write failed");
    }
  }
  if (h.sv_bytes) {
    if (!c->sv) {
      int rc = dev_alloc(c, reinterpret_cast<void**>(&c->sv), (size_t)h.sv_bytes, "cudaMalloc(viscous rate)");
      if (rc) {
        fclose(f);
        return rc;
      }
    }
    if (fread(host.data(), 1, h.sv_bytes, f) != h.sv_bytes) return io_fail(f, "truncated state file");
    if (cudaMemcpy(c->sv, host.data(), h.sv_bytes, cudaMemcpyHostToDevice) != cudaSuccess) return io_fail(f, "device write failed");
  } else if (c->sv) {
    cudaFree(c->sv);
    c->bytes -= (uint64_t)c->plane * sizeof(float);
    c->sv = nullptr;
  }
  fclose(f);
  c->het = h.het != 0;
  c->cur = h.cur;
  c->steps = h.steps;
  c->history = h.history;
  c->init_p0 = h.init_p0;
  c->init_ux = h.init_ux;
  c->init_uy = h.init_uy;
  c->init_phip = h.init_phip;
  // the file's parameters (walls, rates, medium constants) replace the context's
  cfg.stream = c->cfg.stream;
  c->cfg = cfg;
  fill_base(c);
  float w[8];
  for (int i = 0; i < 8; ++i) w[i] = (float)cfg.u_wall[i / 2][i % 2];
  LBM_CUDA(cudaMemcpy(c->walls, w, sizeof(w), cudaMemcpyHostToDevice), "copy of wall velocities");
  return LBM_OK;
}

int lbm_sync(lbm_ctx* c) {
  if (!c) return fail(LBM_EINVAL, "null context");
  LBM_CUDA(cudaGetLastError(), "pending launch error");
  return check_error_word(c);
}

int lbm_step_count(const lbm_ctx* c, int64_t* steps) {
  if (!c || !steps) return fail(LBM_EINVAL, "null argument");
  *steps = c->steps;
  return LBM_OK;
}

int lbm_memory_bytes(const lbm_ctx* c, uint64_t* bytes) {
  if (!c || !bytes) return fail(LBM_EINVAL, "null argument");
  *bytes = c->bytes;
  return LBM_OK;
}

const char* lbm_strerror(int code) {
  switch (code) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "unstable: non-finite velocity";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_EABI: return "ABI version mismatch";
    case LBM_ESTATE: return "invalid state for this call";
    default: return "unknown error";
  }
}

const char* lbm_last_error(void) { return g_msg; }

}  // extern "C"
