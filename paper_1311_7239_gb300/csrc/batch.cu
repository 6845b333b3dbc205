// Batched ensembles: many independent lattices (each with its own size, boundaries, medium and
// parameters) advanced together by one persistent launch per time step.
//
// Memory: the population buffers of all lattices live in two pools (A-B streaming for the whole
// batch), each lattice's planes at its own offset with its own pitch; the medium fields and
// wall velocities likewise.  With in-place streaming (every lattice LBM_STREAM_INPLACE) there is one
// pool, each lattice's buffer laid out as for a single in-place context (ghost rows and column),
// and one CTA per work item of the in-place step.  Per step, the work items of all lattices (frame groups and row
// chunks, exactly as for a single lattice) are concatenated and either one CTA per item (k = 0,
// with a per-item lattice table) or a persistent grid of SMs x k CTAs walks them; the CTA size
// and k are tuning parameters (lbm_batch_tune times the choices on the live batch).
#include <math.h>
#include <string.h>

#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

constexpr int kBatchGraphSteps = 32;

int fail_msg(int code, const char* msg) { return record_error(code, msg); }

#define LBM_BCUDA(call, what)                                                 \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess)                                                    \
      return fail_msg(e_ == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, what); \
  } while (0)

}  // namespace

struct lbm_batch {
  int n = 0;
  int prec = PREC_FP32;
  size_t elem = 4;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<lbm_config> cfg;
  std::vector<int> pitch;
  std::vector<int64_t> plane, foff, moff;
  void* pool[2] = {nullptr, nullptr};
  bool inplace = false;
  int64_t pool_elems = 0;  // elements of one pool
  float* phi = nullptr;
  float* K = nullptr;
  float* walls = nullptr;
  unsigned int* err = nullptr;
  float* stage = nullptr;
  size_t stage_bytes = 0;
  std::vector<StepParams> hp[2];
  StepParams* dp[2] = {nullptr, nullptr};
  int64_t* item_start = nullptr;
  int* item_lattice = nullptr;  // lattice of each work item (one-CTA-per-item form only)
  int64_t item_lattice_cap = 0;
  int64_t total_items = 0;
  int nt = 128, ctas_per_sm = 4, grid = 0, sms = 0;
  int items_per_cta = 1;  // ctas_per_sm = 0: consecutive work items per CTA (4 x items_per_cta cells per thread)
  int flat = 1;  // tiling of the A-B batched kernel (LBM_TILING_FLAT / LBM_TILING_ROWS)
  // A-B batches whose lattices share rho0, s_e, s_q and the storage scale: per-lattice records of the
  // fields that differ (one array per buffer parity) for the per-item kernel
  bool shared_consts = false;
  BatchRec* rec[2] = {nullptr, nullptr};
  int cur = 0;
  int64_t steps = 0;
  int64_t cells = 0;
  uint64_t bytes = 0;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t capture_stream = nullptr;
};

namespace {

int balloc(lbm_batch* b, void** p, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return fail_msg(e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA, what);
  }
  b->bytes += bytes;
  return LBM_OK;
}

void drop_graphs(lbm_batch* b) {
  for (int k = 0; k < 2; ++k) {
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
    b->graph[k] = nullptr;
  }
}

void release(lbm_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  for (int k = 0; k < 2; ++k) {
    cudaFree(b->pool[k]);
    cudaFree(b->dp[k]);
    cudaFree(b->rec[k]);
  }
  cudaFree(b->phi);
  cudaFree(b->K);
  cudaFree(b->walls);
  cudaFree(b->err);
  cudaFree(b->stage);
  cudaFree(b->item_start);
  cudaFree(b->item_lattice);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

// Parameters of lattice d when buffer `cur` holds its current state.
StepParams params_of(const lbm_batch* b, int d, int cur) { return b->hp[cur][d]; }

int set_launch(lbm_batch* b, int nt, int ctas_per_sm) {
  if (nt != 64 && nt != 128 && nt != 256) return fail_msg(LBM_EINVAL, "threads per CTA must be 64, 128 or 256");
  if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail_msg(LBM_EINVAL, "CTAs per SM must be in [0, 32]");
  if (b->inplace && (nt != 128 || ctas_per_sm != 0))
    return fail_msg(LBM_EINVAL, "in-place batches run one CTA of 128 threads per work item (launch shape 128, 0)");
  std::vector<int64_t> start(b->n);
  int64_t total = 0;
  for (int d = 0; d < b->n; ++d) {
    start[d] = total;
    const lbm_config& c = b->cfg[d];
    total += b->inplace ? inplace_items((int)c.nx, (int)c.ny, (int)c.bc_x, (int)c.bc_y)
                        : batch_items((int)c.nx, (int)c.ny, (int)c.bc_y, nt, b->flat);
  }
  LBM_BCUDA(cudaMemcpy(b->item_start, start.data(), b->n * sizeof(int64_t), cudaMemcpyHostToDevice), "copy of the item table");
  b->total_items = total;
  b->nt = nt;
  drop_graphs(b);
  if (ctas_per_sm == 0 && b->items_per_cta > 1) {  // CTAs of items_per_cta consecutive items (the range walk)
    const int64_t g = (total + b->items_per_cta - 1) / b->items_per_cta;
    if (g > 0x7fffffffLL) return fail_msg(LBM_EINVAL, "too many work items for the grid");
    b->ctas_per_sm = 0;
    b->grid = (int)g;
    return LBM_OK;
  }
  if (ctas_per_sm == 0) {  // one CTA per work item
    if (total > 0x7fffffffLL) return fail_msg(LBM_EINVAL, "too many work items for one CTA per item");
    if (b->item_lattice_cap < total) {
      cudaStreamSynchronize(b->stream);
      cudaFree(b->item_lattice);
      b->bytes -= (uint64_t)b->item_lattice_cap * sizeof(int);
      b->item_lattice = nullptr;
      b->item_lattice_cap = 0;
      int rc = balloc(b, reinterpret_cast<void**>(&b->item_lattice), (size_t)total * sizeof(int), "cudaMalloc(item lattice table)");
      if (rc) return rc;
      b->item_lattice_cap = total;
    }
    std::vector<int> lat((size_t)total);
    for (int d = 0; d < b->n; ++d) {
      const int64_t e = d + 1 < b->n ? start[d + 1] : total;
      for (int64_t i = start[d]; i < e; ++i) lat[(size_t)i] = d;
    }
    LBM_BCUDA(cudaMemcpy(b->item_lattice, lat.data(), (size_t)total * sizeof(int), cudaMemcpyHostToDevice), "copy of the item lattice table");
    b->ctas_per_sm = 0;
    b->grid = (int)total;
    return LBM_OK;
  }
  // persistent CTAs must all be resident: no more per SM than the kernel's occupancy allows
  const int kmax = batch_max_ctas_per_sm(b->prec, nt);
  if (ctas_per_sm > kmax) ctas_per_sm = kmax;
  b->ctas_per_sm = ctas_per_sm;
  const int64_t g = (int64_t)b->sms * ctas_per_sm;
  b->grid = (int)(g < total ? g : total);
  return LBM_OK;
}

// One batched step from buffer parity `cur` on stream s, in the form the launch shape selects.
cudaError_t launch_batch(const lbm_batch* b, int cur, cudaStream_t s) {
  if (b->inplace)
    return launch_step_batch_inplace(b->dp[cur], b->item_start, b->item_lattice, b->total_items, b->prec, cur, s);
  const bool per_item = b->ctas_per_sm == 0 && b->items_per_cta == 1;
  if (b->shared_consts && per_item)
    return launch_step_batch_shared(b->hp[0][0], b->rec[cur], b->dp[cur], b->item_start, b->item_lattice, b->total_items, b->prec,
                                    b->nt, b->flat, s);
  // otherwise the range walk: a persistent grid, or ceil(items / items_per_cta) CTAs
  return launch_step_batch(b->dp[cur], b->item_start, per_item ? b->item_lattice : nullptr, b->n, b->total_items, b->prec, b->nt,
                           b->grid, b->flat, s);
}

int launch_once(lbm_batch* b, int cur, cudaStream_t s) {
  LBM_BCUDA(launch_batch(b, cur, s), "batched step kernel");
  return LBM_OK;
}

int capture(lbm_batch* b, int cur) {
  if (!b->capture_stream) LBM_BCUDA(cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking), "cudaStreamCreate");
  LBM_BCUDA(cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < kBatchGraphSteps && le == cudaSuccess; ++k) le = launch_batch(b, cur ^ (k & 1), b->capture_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->capture_stream, &g);
  if (le != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail_msg(LBM_ECUDA, "capture of the batched step graph");
  }
  e = cudaGraphInstantiate(&b->graph[cur], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph[cur] = nullptr;
    return fail_msg(LBM_ECUDA, "cudaGraphInstantiate");
  }
  return LBM_OK;
}

int check_index(const lbm_batch* b, int d) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (d < 0 || d >= b->n) return fail_msg(LBM_EINVAL, "lattice index out of range");
  return LBM_OK;
}

bool on_device(const lbm_batch* b, const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == b->device;
}

int ensure_stage(lbm_batch* b, size_t bytes) {
  if (b->stage_bytes >= bytes) return LBM_OK;
  if (b->stage) {
    cudaStreamSynchronize(b->stream);
    cudaFree(b->stage);
    b->bytes -= b->stage_bytes;
    b->stage = nullptr;
    b->stage_bytes = 0;
  }
  int rc = balloc(b, reinterpret_cast<void**>(&b->stage), bytes, "cudaMalloc(staging)");
  if (rc == LBM_OK) b->stage_bytes = bytes;
  return rc;
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_config* cfgs, int n, lbm_batch** out) {
  if (!cfgs || !out || n < 1) return fail_msg(LBM_EINVAL, "lbm_batch_create: need n >= 1 configurations");
  *out = nullptr;
  for (int d = 0; d < n; ++d) {
    int rc = validate_config(&cfgs[d]);
    if (rc) return rc;
    if (cfgs[d].thermal) return fail_msg(LBM_EINVAL, "lbm_batch_create: batches hold isothermal lattices only");
    if (cfgs[d].streaming != cfgs[0].streaming) return fail_msg(LBM_EINVAL, "lbm_batch_create: all lattices need one streaming form");
    if (cfgs[d].streaming == LBM_STREAM_INPLACE && (cfgs[d].bc_x > LBM_WALL || cfgs[d].bc_y > LBM_WALL))
      return fail_msg(LBM_EINVAL, "lbm_batch_create: in-place batches take periodic and halfway-wall sides only");
    if (cfgs[d].precision != cfgs[0].precision) return fail_msg(LBM_EINVAL, "lbm_batch_create: all lattices need one precision");
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return fail_msg(LBM_ENOMEM, "host allocation of the batch");
  b->n = n;
  b->cfg.assign(cfgs, cfgs + n);
  b->prec = (int)cfgs[0].precision;
  b->elem = b->prec == PREC_FP32 ? 4 : 2;
  b->inplace = cfgs[0].streaming == LBM_STREAM_INPLACE;
  if (cudaGetDevice(&b->device) != cudaSuccess || cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    delete b;
    return fail_msg(LBM_ECUDA, "no usable current device");
  }
  if (cfgs[0].stream) {
    b->stream = static_cast<cudaStream_t>(cfgs[0].stream);
  } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return fail_msg(LBM_ECUDA, "cudaStreamCreate");
  } else {
    b->own_stream = true;
  }
  b->pitch.resize(n);
  b->plane.resize(n);
  b->foff.resize(n);
  b->moff.resize(n);
  int64_t fel = 0, mel = 0;
  for (int d = 0; d < n; ++d) {
    b->pitch[d] = (int)((cfgs[d].nx + 127) / 128 * 128);
    b->plane[d] = (int64_t)b->pitch[d] * (cfgs[d].ny + (b->inplace ? 2 : 0));
    b->foff[d] = fel;
    b->moff[d] = mel;
    // in-place: the planes with their ghost rows, then the ghost column (rounded to 128 elements
    // so that the next lattice's rows stay aligned); the step indexes a buffer with 32-bit offsets
    const int64_t buf = b->inplace ? (8 * (b->plane[d] + cfgs[d].ny + 2) + 127) / 128 * 128 : 8 * b->plane[d];
    if (b->inplace && buf > (1ll << 32)) {
      if (b->own_stream) cudaStreamDestroy(b->stream);
      delete b;
      return fail_msg(LBM_EINVAL, "lbm_batch_create: an in-place lattice needs 8 ((ny + 2) pitch + ny + 2) <= 2^32 elements");
    }
    fel += buf;
    mel += b->plane[d];
    b->cells += (int64_t)cfgs[d].nx * cfgs[d].ny;
  }
  b->pool_elems = fel;
  int rc = LBM_OK;
  for (int k = 0; k < (b->inplace ? 1 : 2) && rc == LBM_OK; ++k) rc = balloc(b, &b->pool[k], fel * b->elem, "cudaMalloc(population pools)");
  if (rc == LBM_OK) rc = balloc(b, reinterpret_cast<void**>(&b->phi), mel * sizeof(float), "cudaMalloc(porosity pool)");
  if (rc == LBM_OK) rc = balloc(b, reinterpret_cast<void**>(&b->K), mel * sizeof(float), "cudaMalloc(permeability pool)");
  if (rc == LBM_OK) rc = balloc(b, reinterpret_cast<void**>(&b->walls), 8 * n * sizeof(float), "cudaMalloc(walls)");
  if (rc == LBM_OK) rc = balloc(b, reinterpret_cast<void**>(&b->err), sizeof(unsigned int), "cudaMalloc(error word)");
  if (rc == LBM_OK) rc = balloc(b, reinterpret_cast<void**>(&b->item_start), n * sizeof(int64_t), "cudaMalloc(item table)");
  for (int k = 0; k < 2 && rc == LBM_OK; ++k) rc = balloc(b, reinterpret_cast<void**>(&b->dp[k]), n * sizeof(StepParams), "cudaMalloc(params)");
  if (rc != LBM_OK) {
    release(b);
    return rc;
  }
  std::vector<float> w(8 * (size_t)n);
  for (int d = 0; d < n; ++d)
    for (int i = 0; i < 8; ++i) w[8 * d + i] = (float)cfgs[d].u_wall[i / 2][i % 2];
  cudaError_t e = cudaMemcpy(b->walls, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(unsigned int), b->stream);
  for (int k = 0; k < (b->inplace ? 1 : 2) && e == cudaSuccess; ++k) e = cudaMemsetAsync(b->pool[k], 0, fel * b->elem, b->stream);
  if (e != cudaSuccess) {
    release(b);
    return fail_msg(LBM_ECUDA, "batch set-up copies");
  }
  char* pool0 = static_cast<char*>(b->pool[0]);
  char* pool1 = static_cast<char*>(b->pool[1]);
  for (int k = 0; k < 2; ++k) b->hp[k].resize(n);
  for (int d = 0; d < n; ++d) {
    StepParams P;
    params_from_config(cfgs[d], b->prec, b->pitch[d], b->plane[d], P);
    P.uw = b->walls + 8 * d;
    P.err = b->err;
    P.phi = b->phi + b->moff[d];
    P.K = b->K + b->moff[d];
    if (b->inplace) {  // one buffer from its row 0; the parity selects the slots
      void* A = pool0 + (b->foff[d] + b->pitch[d]) * b->elem;
      P.inplace = 1;
      for (int k = 0; k < 2; ++k) {
        b->hp[k][d] = P;
        b->hp[k][d].src = b->hp[k][d].dst = A;
        b->hp[k][d].parity = k;
      }
    } else {
      void* A = pool0 + b->foff[d] * b->elem;
      void* B = pool1 + b->foff[d] * b->elem;
      b->hp[0][d] = P;
      b->hp[0][d].src = A;
      b->hp[0][d].dst = B;
      b->hp[1][d] = P;
      b->hp[1][d].src = B;
      b->hp[1][d].dst = A;
    }
    // every lattice keeps per-cell medium fields, filled with its uniform values until set
    e = launch_medium(nullptr, nullptr, (float)cfgs[d].phi, (float)cfgs[d].K, (int)cfgs[d].nx, (int)cfgs[d].ny, b->pitch[d],
                      b->phi + b->moff[d], b->K + b->moff[d], b->err, 0, b->stream);
    if (e != cudaSuccess) break;
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaMemcpyAsync(b->dp[k], b->hp[k].data(), n * sizeof(StepParams), cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) {
    release(b);
    return fail_msg(LBM_ECUDA, "batch parameter upload");
  }
  // the per-lattice records of A-B batches whose lattices share the collision constants (the
  // in-place kernel passes its parameters on to an out-of-line frame function, which would keep a
  // per-CTA copy in local memory: 79.7 -> 47.3 GLUPS, so in-place batches keep the staged form)
  bool shared = !b->inplace;
  for (int d = 1; d < n && shared; ++d)
    shared = cfgs[d].rho0 == cfgs[0].rho0 && cfgs[d].s_e == cfgs[0].s_e && cfgs[d].s_q == cfgs[0].s_q &&
             b->hp[0][d].scale == b->hp[0][0].scale;
  if (shared) {
    std::vector<BatchRec> r(n);
    for (int k = 0; k < 2 && rc == LBM_OK && e == cudaSuccess; ++k) {
      for (int d = 0; d < n; ++d) {
        const StepParams& P = b->hp[k][d];
        r[d] = BatchRec{P.src, P.dst, P.phi, P.K, P.uw, P.plane, P.nx, P.ny, P.pitch, P.bc_x, P.bc_y, P.forch, P.nu, P.s_v, P.ax, P.ay};
      }
      rc = balloc(b, reinterpret_cast<void**>(&b->rec[k]), n * sizeof(BatchRec), "cudaMalloc(lattice records)");
      if (rc == LBM_OK) e = cudaMemcpy(b->rec[k], r.data(), n * sizeof(BatchRec), cudaMemcpyHostToDevice);
    }
    if (rc != LBM_OK || e != cudaSuccess) {
      release(b);
      return rc != LBM_OK ? rc : fail_msg(LBM_ECUDA, "batch record upload");
    }
    b->shared_consts = true;
  }
  if ((rc = set_launch(b, b->inplace ? 128 : 64, 0)) || (rc = lbm_batch_init_equilibrium(b, -1, 1.0, 0.0, 0.0, 0))) {
    release(b);
    return rc;
  }
  *out = b;
  return LBM_OK;
}

int lbm_create_batch(const lbm_config* cfgs, int n, lbm_batch** out) { return lbm_batch_create(cfgs, n, out); }

void lbm_batch_destroy(lbm_batch* b) { release(b); }

int lbm_batch_set_medium(lbm_batch* b, int d, const float* eps, const float* K) {
  int rc = check_index(b, d);
  if (rc) return rc;
  const size_t n = (size_t)b->cfg[d].nx * b->cfg[d].ny;
  const float* de = eps;
  const float* dk = K;
  if ((eps && !on_device(b, eps)) || (K && !on_device(b, K))) {
    if ((rc = ensure_stage(b, 2 * n * sizeof(float)))) return rc;
    if (eps && !on_device(b, eps)) {
      LBM_BCUDA(cudaMemcpyAsync(b->stage, eps, n * sizeof(float), cudaMemcpyHostToDevice, b->stream), "copy of eps");
      de = b->stage;
    }
    if (K && !on_device(b, K)) {
      LBM_BCUDA(cudaMemcpyAsync(b->stage + n, K, n * sizeof(float), cudaMemcpyHostToDevice, b->stream), "copy of K");
      dk = b->stage + n;
    }
  }
  const StepParams& P = b->hp[0][d];
  LBM_BCUDA(cudaMemsetAsync(b->err, 0, sizeof(unsigned int), b->stream), "cudaMemset");
  LBM_BCUDA(launch_medium(de, dk, (float)b->cfg[d].phi, (float)b->cfg[d].K, P.nx, P.ny, P.pitch, const_cast<float*>(P.phi),
                          const_cast<float*>(P.K), b->err, 0, b->stream),
            "medium kernel");
  unsigned int h = 0;
  LBM_BCUDA(cudaMemcpyAsync(&h, b->err, sizeof(h), cudaMemcpyDeviceToHost, b->stream), "read of error word");
  LBM_BCUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (h & 2u) {
    cudaMemsetAsync(b->err, 0, sizeof(unsigned int), b->stream);
    return fail_msg(LBM_EINVAL, "medium out of range: need 0 < eps <= 1 and 0 < K < 3e38");
  }
  return LBM_OK;
}

int lbm_batch_init_equilibrium(lbm_batch* b, int d, double p0, double ux0, double uy0, int phi_p_uniform) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (d < -1 || d >= b->n) return fail_msg(LBM_EINVAL, "lattice index out of range");
  const int lo = d < 0 ? 0 : d, hi = d < 0 ? b->n : d + 1;
  for (int k = lo; k < hi; ++k) {
    StepParams P = params_of(b, k, b->cur);
    if (b->inplace) {
      LBM_BCUDA(launch_put_inplace(P, b->prec, true, nullptr, nullptr, true, false, (float)p0, (float)ux0, (float)uy0,
                                   phi_p_uniform ? 1 : 0, 0.0f, b->stream),
                "init kernel");
      continue;
    }
    P.dst = const_cast<void*>(P.src);  // the init writes the current buffer
    LBM_BCUDA(launch_init(P, b->prec, true, false, (float)p0, (float)ux0, (float)uy0, phi_p_uniform ? 1 : 0, 0.0f, true, false,
                          b->stream),
              "init kernel");
  }
  if (d < 0) b->steps = 0;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int n) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (n < 0) return fail_msg(LBM_EINVAL, "negative step count");
  while (n >= kBatchGraphSteps) {
    if (!b->graph[b->cur]) {
      int rc = capture(b, b->cur);
      if (rc) return rc;
    }
    LBM_BCUDA(cudaGraphLaunch(b->graph[b->cur], b->stream), "cudaGraphLaunch");
    b->steps += kBatchGraphSteps;
    n -= kBatchGraphSteps;
  }
  for (int k = 0; k < n; ++k) {
    int rc = launch_once(b, b->cur, b->stream);
    if (rc) return rc;
    b->cur ^= 1;
    ++b->steps;
  }
  return LBM_OK;
}

int lbm_batch_step_each(lbm_batch* b, int n) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (n < 0) return fail_msg(LBM_EINVAL, "negative step count");
  for (int d = 0; d < b->n; ++d) {
    int cur = b->cur;
    for (int k = 0; k < n; ++k) {
      const StepParams P = params_of(b, d, cur);
      LBM_BCUDA(b->inplace ? launch_step_inplace(P, b->prec, true, false, b->stream) : launch_step(P, b->prec, true, false, b->stream),
                "step kernel");
      cur ^= 1;
    }
  }
  b->cur ^= (n & 1);
  b->steps += n;
  return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch* b, int threads_per_cta, int ctas_per_sm) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  return set_launch(b, threads_per_cta, ctas_per_sm);
}

int lbm_batch_get_launch(const lbm_batch* b, int* threads_per_cta, int* ctas_per_sm) {
  if (!b || !threads_per_cta || !ctas_per_sm) return fail_msg(LBM_EINVAL, "null argument");
  *threads_per_cta = b->nt;
  *ctas_per_sm = b->ctas_per_sm;
  return LBM_OK;
}

int lbm_batch_set_items_per_cta(lbm_batch* b, int items_per_cta) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (items_per_cta != 1 && items_per_cta != 2 && items_per_cta != 4 && items_per_cta != 8)
    return fail_msg(LBM_EINVAL, "work items per CTA must be 1, 2, 4 or 8");
  if (b->inplace && items_per_cta != 1) return fail_msg(LBM_EINVAL, "in-place batches run one work item per CTA");
  const int old = b->items_per_cta;
  b->items_per_cta = items_per_cta;
  const int rc = set_launch(b, b->nt, b->ctas_per_sm);
  if (rc) b->items_per_cta = old;
  return rc;
}

int lbm_batch_get_items_per_cta(const lbm_batch* b, int* items_per_cta) {
  if (!b || !items_per_cta) return fail_msg(LBM_EINVAL, "null argument");
  *items_per_cta = b->items_per_cta;
  return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch* b, int tiling) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (tiling != LBM_TILING_ROWS && tiling != LBM_TILING_FLAT) return fail_msg(LBM_EINVAL, "tiling must be LBM_TILING_ROWS or LBM_TILING_FLAT");
  if (b->inplace && tiling != LBM_TILING_FLAT) return fail_msg(LBM_EINVAL, "in-place batches keep their own tiling (LBM_TILING_FLAT)");
  if (b->inplace) return LBM_OK;
  const int old = b->flat;
  b->flat = tiling == LBM_TILING_FLAT ? 1 : 0;
  const int rc = set_launch(b, b->nt, b->ctas_per_sm);
  if (rc) b->flat = old;
  return rc;
}

int lbm_batch_get_tiling(const lbm_batch* b, int* tiling) {
  if (!b || !tiling) return fail_msg(LBM_EINVAL, "null argument");
  *tiling = b->flat ? LBM_TILING_FLAT : LBM_TILING_ROWS;
  return LBM_OK;
}

int lbm_batch_tune(lbm_batch* b, int steps, int* threads_per_cta, int* ctas_per_sm, float* ms_per_step) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (steps < 1) return fail_msg(LBM_EINVAL, "steps must be positive");
  // time every choice on a copy of the current state, then restore it (in-place batches have one)
  const size_t pool_bytes = (size_t)b->pool_elems * b->elem;
  void* save = nullptr;
  LBM_BCUDA(cudaMalloc(&save, pool_bytes), "cudaMalloc(tuning copy)");
  void* live = b->pool[b->inplace ? 0 : b->cur];
  cudaMemcpyAsync(save, live, pool_bytes, cudaMemcpyDeviceToDevice, b->stream);
  const int nts[3] = {64, 128, 256};
  // (CTAs per SM, work items per CTA): one CTA per item, CTAs of 2 and 4 consecutive items (8 and
  // 16 cells per thread), persistent grids of SMs x k CTAs
  const int ks[8] = {0, 0, 0, 1, 2, 4, 8, 16};
  const int ipc[8] = {1, 2, 4, 1, 1, 1, 1, 1};
  const int n_nt = b->inplace ? 1 : 3, n_k = b->inplace ? 1 : 8;
  const int* nt_list = b->inplace ? &nts[1] : nts;
  const int n_tiling = b->inplace ? 1 : 2;  // flat, then rows
  float best = 1e30f;
  int best_nt = b->nt, best_k = b->ctas_per_sm, best_flat = b->flat, best_ipc = b->items_per_cta;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = LBM_OK;
  for (int f = 0; f < n_tiling && rc == LBM_OK; ++f)
  for (int a = 0; a < n_nt && rc == LBM_OK; ++a)
    for (int c = 0; c < n_k && rc == LBM_OK; ++c) {
      if (ks[c] > batch_max_ctas_per_sm(b->prec, nt_list[a])) continue;  // persistent CTAs must be resident
      b->flat = b->inplace || f == 0 ? 1 : 0;
      b->items_per_cta = ipc[c];
      if ((rc = set_launch(b, nt_list[a], ks[c]))) break;
      if ((rc = launch_once(b, b->cur, b->stream))) break;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int s = 0; s < steps && rc == LBM_OK; ++s) rc = launch_once(b, b->cur ^ ((s + 1) & 1), b->stream);
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= steps;
      if (ms < best) {
        best = ms;
        best_nt = nt_list[a];
        best_k = ks[c];
        best_flat = b->flat;
        best_ipc = ipc[c];
      }
    }
  cudaMemcpyAsync(live, save, pool_bytes, cudaMemcpyDeviceToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  b->flat = best_flat;
  b->items_per_cta = best_ipc;
  if ((rc = set_launch(b, best_nt, best_k))) return rc;
  if (threads_per_cta) *threads_per_cta = best_nt;
  if (ctas_per_sm) *ctas_per_sm = best_k;
  if (ms_per_step) *ms_per_step = best;
  return LBM_OK;
}

int lbm_batch_macros(lbm_batch* b, int d, float* p, float* ux, float* uy) {
  int rc = check_index(b, d);
  if (rc) return rc;
  const size_t n = (size_t)b->cfg[d].nx * b->cfg[d].ny;
  float* outs[3] = {p, ux, uy};
  float* dev[3] = {p, ux, uy};
  bool host = false;
  for (int i = 0; i < 3; ++i)
    if (outs[i] && !on_device(b, outs[i])) host = true;
  if (host && (rc = ensure_stage(b, 3 * n * sizeof(float)))) return rc;
  for (int i = 0; i < 3; ++i)
    if (outs[i] && !on_device(b, outs[i])) dev[i] = b->stage + i * n;
  LBM_BCUDA(launch_macros(params_of(b, d, b->cur), b->prec, true, false, dev[0], dev[1], dev[2], nullptr, b->stream), "macros kernel");
  for (int i = 0; i < 3; ++i)
    if (outs[i] && dev[i] != outs[i])
      LBM_BCUDA(cudaMemcpyAsync(outs[i], dev[i], n * sizeof(float), cudaMemcpyDeviceToHost, b->stream), "copy of output");
  if (host) LBM_BCUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  return LBM_OK;
}

int lbm_batch_get_populations(lbm_batch* b, int d, float* f) {
  int rc = check_index(b, d);
  if (rc) return rc;
  if (!f) return fail_msg(LBM_EINVAL, "null output");
  const size_t n = (size_t)b->cfg[d].nx * b->cfg[d].ny;
  float* dev = f;
  const bool host = !on_device(b, f);
  if (host) {
    if ((rc = ensure_stage(b, 8 * n * sizeof(float)))) return rc;
    dev = b->stage;
  }
  LBM_BCUDA(launch_export(params_of(b, d, b->cur), b->prec, true, false, dev, nullptr, b->stream), "export kernel");
  if (host) {
    LBM_BCUDA(cudaMemcpyAsync(f, dev, 8 * n * sizeof(float), cudaMemcpyDeviceToHost, b->stream), "copy of output");
    LBM_BCUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  }
  return LBM_OK;
}

int lbm_batch_info(const lbm_batch* b, int64_t* cells, int64_t* steps, uint64_t* bytes) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  if (cells) *cells = b->cells;
  if (steps) *steps = b->steps;
  if (bytes) *bytes = b->bytes;
  return LBM_OK;
}

int lbm_batch_sync(lbm_batch* b) {
  if (!b) return fail_msg(LBM_EINVAL, "null batch");
  unsigned int h = 0;
  LBM_BCUDA(cudaGetLastError(), "pending launch error");
  LBM_BCUDA(cudaMemcpyAsync(&h, b->err, sizeof(h), cudaMemcpyDeviceToHost, b->stream), "read of error word");
  LBM_BCUDA(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (h & 4u) return fail_msg(LBM_ECUDA, "a kernel index left its buffer (debug build check)");
  if (h & 1u) return fail_msg(LBM_EUNSTABLE, "a lattice of the batch produced a non-finite velocity");
  return LBM_OK;
}

}  // extern "C"
