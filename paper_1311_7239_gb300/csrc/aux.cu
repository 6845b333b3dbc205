// Set-up and read-out kernels around the fused step: medium upload and checks, equilibrium
// initial state (Sec. 3.1: moments at equilibrium, u = u0, p = p0), population import/export,
// macroscopic fields (Eqs. 18-20, T = sum g), the FP64 steady-state residual and the hot/cold wall
// Nusselt number (Sec. 3.4, Table 1).
//
// The stored state is post-collision (pull streaming).  Read-outs therefore gather first: the
// pre-collision populations of the paper's f(x, t) are the gathered values, and importing a
// pre-collision state scatters it back into the slots the next gather reads.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

// --------------------------------------------------------------------------------------------
// medium: dense [ny][nx] user arrays -> pitched fields, with range checks (err bit 1)
// --------------------------------------------------------------------------------------------
__global__ void k_medium(const float* __restrict__ eps, const float* __restrict__ K, float phi_u, float K_u, int nx, int ny,
                         int pitch, float* __restrict__ phi_out, float* __restrict__ K_out, unsigned int* err, int log_k) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (y >= ny) return;
  const int64_t o = (int64_t)y * pitch + x;
  if (x >= nx) {  // padding: harmless values
    if (x < pitch) { phi_out[o] = 1.0f; K_out[o] = 1.0f; }
    return;
  }
  const int64_t i = (int64_t)y * nx + x;
  const float ph = eps ? eps[i] : phi_u;
  const float k = K ? (log_k ? expf(K[i]) : K[i]) : K_u;
  if (!(ph > 0.0f && ph <= 1.0f) || !(k > 0.0f && k < 3.0e38f)) atomicOr(err, 2u);
  phi_out[o] = ph;
  K_out[o] = k;
}

// viscous rate field from a viscosity-ratio field: s_v = 1 / (1/2 + J nu / c_s^2) (Eq. 21, Sec. 3.2)
__global__ void k_viscous_rate(const float* __restrict__ J, int nx, int ny, int pitch, float nu, float* __restrict__ sv,
                               unsigned int* err) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (y >= ny || x >= pitch) return;
  const int64_t o = (int64_t)y * pitch + x;
  if (x >= nx) {
    sv[o] = 1.0f;
    return;
  }
  const float j = J[(int64_t)y * nx + x];
  if (!(j > 0.0f && j < 1e30f)) atomicOr(err, 2u);
  sv[o] = 1.0f / (0.5f + 3.0f * j * nu);
}

cudaError_t launch_viscous_rate(const float* J, int nx, int ny, int pitch, float nu, float* sv, unsigned int* err, cudaStream_t s) {
  k_viscous_rate<<<dim3((pitch + 255) / 256, ny), 256, 0, s>>>(J, nx, ny, pitch, nu, sv, err);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------------------------
// helpers for the inverse of the gather
// --------------------------------------------------------------------------------------------
// Where a slot s_j(x) goes: the cell x + e_j if that is inside (after periodic wrap), else the
// cell x itself through bounce-back into direction opp(j).
__device__ __forceinline__ bool slot_target(const StepParams& P, int x, int y, int ex, int ey, int& tx, int& ty) {
  tx = x + ex;
  ty = y + ey;
  if (P.bc_x != BC_WALL) tx = (tx + P.nx) % P.nx;
  if (P.bc_y != BC_WALL) ty = (ty + P.ny) % P.ny;
  return tx >= 0 && tx < P.nx && ty >= 0 && ty < P.ny;
}

// pre-collision deviation of equilibrium (Eq. 22) at cell (x, y)
template <bool HET>
__device__ __forceinline__ void feq_cell(const StepParams& P, int x, int y, float p0, float ux0, float uy0, int phip_uniform,
                                         float out[8]) {
  const Coef c = coef_at<HET>(P, x, y);
  const float phip = phip_uniform ? p0 : c.phi * p0;
  feq_dev_d2q8(phip - P.p_rest, ux0, uy0, c.inv_phi, P.rho0, out);
}

template <int PREC, bool HET>
__global__ void k_init_flow(const StepParams P, float p0, float ux0, float uy0, int phip_uniform) {
  using S = Store<PREC>;
  using T = typename S::T;
  T* dst = static_cast<T*>(P.dst);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.pitch) return;
  const int64_t r = (int64_t)y * P.pitch + x;
  if (x >= P.nx) {
    for (int j = 0; j < 8; ++j) dst[j * P.plane + r] = S::enc(0.0f, P.scale);
    return;
  }
  float own[8];
  feq_cell<HET>(P, x, y, p0, ux0, uy0, phip_uniform, own);
#pragma unroll 1
  for (int j = 0; j < 8; ++j) {
    int tx, ty;
    float v;
    if (slot_target(P, x, y, ex_of(j), ey_of(j), tx, ty)) {
      float nb[8];
      feq_cell<HET>(P, tx, ty, p0, ux0, uy0, phip_uniform, nb);
      v = nb[j];
    } else {
      const int w = wall_of(tx, ty, P.ny);
      v = own[opp_of(j)] + 6.0f * w_of(j) * P.rho0 * ((float)ex_of(j) * P.uw[2 * w] + (float)ey_of(j) * P.uw[2 * w + 1]);
    }
    dst[j * P.plane + r] = S::enc(v, P.scale);
  }
}

// Inverse of the temperature gather for one slot, given the pre-collision deviations z of the
// target cell (inside) or of the own cell (wall).
__device__ __forceinline__ float g_slot(const StepParams& P, int x, int y, int j, const float* z_own, const float* z_tgt,
                                        bool inside, int w) {
  if (j == 0 || inside) return z_tgt[j];
  const float zo = z_own[opp5(j)];
  return P.Tdir[w] ? (-zo + 0.4f * (P.Tw[w] - P.T0)) : zo;
  (void)x; (void)y;
}

template <int PREC>
__global__ void k_init_thermal(const StepParams P, float T_init, float ux0, float uy0) {
  using S = Store<PREC>;
  using T = typename S::T;
  T* gdst = static_cast<T*>(P.gdst);
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.pitch) return;
  const int64_t r = (int64_t)y * P.pitch + x;
  float z[5];
  geq_dev(P, T_init, ux0, uy0, z);  // uniform state: every cell has the same z
  for (int j = 0; j < 5; ++j) {
    float v = 0.0f;
    if (x < P.nx) {
      int tx, ty;
      const bool inside = j == 0 || slot_target(P, x, y, ex5(j), ey5(j), tx, ty);
      const int w = inside ? 0 : wall_of(tx, ty, P.ny);
      v = g_slot(P, x, y, j, z, z, inside, w);
    }
    gdst[j * P.plane + r] = S::enc(v, P.scale);
  }
}

// --------------------------------------------------------------------------------------------
// import of a pre-collision state (dense float32 [q][ny][nx], full populations)
// --------------------------------------------------------------------------------------------
template <int PREC>
__global__ void k_import(const StepParams P, const float* __restrict__ f, const float* __restrict__ g) {
  using S = Store<PREC>;
  using T = typename S::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.pitch) return;
  const int64_t r = (int64_t)y * P.pitch + x;
  const int64_t dense = (int64_t)P.nx * P.ny;
  if (f) {
    T* dst = static_cast<T*>(P.dst);
    for (int j = 0; j < 8; ++j) {
      float v = 0.0f;
      if (x < P.nx) {
        int tx, ty;
        if (slot_target(P, x, y, ex_of(j), ey_of(j), tx, ty)) {
          v = f[j * dense + (int64_t)ty * P.nx + tx] - 3.0f * w_of(j) * P.p_rest;
        } else {
          const int w = wall_of(tx, ty, P.ny);
          const int o = opp_of(j);
          v = f[o * dense + (int64_t)y * P.nx + x] - 3.0f * w_of(o) * P.p_rest +
              6.0f * w_of(j) * P.rho0 * ((float)ex_of(j) * P.uw[2 * w] + (float)ey_of(j) * P.uw[2 * w + 1]);
        }
      }
      dst[j * P.plane + r] = S::enc(v, P.scale);
    }
  }
  if (g) {
    T* gdst = static_cast<T*>(P.gdst);
    const float g0 = 0.2f * P.T0;
    for (int j = 0; j < 5; ++j) {
      float v = 0.0f;
      if (x < P.nx) {
        int tx = x, ty = y;
        const bool inside = j == 0 || slot_target(P, x, y, ex5(j), ey5(j), tx, ty);
        if (inside) {
          v = g[j * dense + (int64_t)ty * P.nx + tx] - g0;
        } else {
          const int w = wall_of(tx, ty, P.ny);
          const float zo = g[opp5(j) * dense + (int64_t)y * P.nx + x] - g0;
          v = P.Tdir[w] ? (-zo + 0.4f * (P.Tw[w] - P.T0)) : zo;
        }
      }
      gdst[j * P.plane + r] = S::enc(v, P.scale);
    }
  }
}

// --------------------------------------------------------------------------------------------
// read-outs: pre-collision populations and macroscopic fields of one cell
// --------------------------------------------------------------------------------------------
template <int PREC, bool HET, bool THERMAL>
__device__ __forceinline__ void gather_state(const StepParams& P, const void* src_v, const void* gsrc_v, int x, int y, float d[8],
                                             float gd[5], float& ay_out) {
  using T = typename Store<PREC>::T;
  ay_out = P.ay;
  if (THERMAL) {
    gather_cell_thermal<PREC, HET>(P, static_cast<const T*>(src_v), static_cast<const T*>(gsrc_v), x, y, d, gd);
    ay_out += P.g_beta * (gd[0] + gd[1] + gd[2] + gd[3] + gd[4]);
  } else {
    gather_cell<PREC, HET>(P, static_cast<const T*>(src_v), x, y, d);
  }
}

template <int PREC, bool HET, bool THERMAL>
__global__ void k_export(const StepParams P, float* __restrict__ f, float* __restrict__ g) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  float d[8], gd[5], ay;
  gather_state<PREC, HET, THERMAL>(P, P.src, P.gsrc, x, y, d, gd, ay);
  const int64_t dense = (int64_t)P.nx * P.ny, o = (int64_t)y * P.nx + x;
  if (f)
    for (int i = 0; i < 8; ++i) f[i * dense + o] = d[i] + 3.0f * w_of(i) * P.p_rest;
  if (THERMAL && g)
    for (int i = 0; i < 5; ++i) g[i * dense + o] = gd[i] + 0.2f * P.T0;
}

template <int PREC, bool HET, bool THERMAL>
__global__ void k_macros(const StepParams P, float* __restrict__ p, float* __restrict__ ux, float* __restrict__ uy, float* __restrict__ Tout) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  float d[8], gd[5], ay;
  gather_state<PREC, HET, THERMAL>(P, P.src, P.gsrc, x, y, d, gd, ay);
  const Coef c = coef_at<HET>(P, x, y);
  const Macro m = macro_d2q8(d, c, P.ax, ay, P.rho0);
  const int64_t o = (int64_t)y * P.nx + x;
  if (p) p[o] = (P.p_rest + m.phip_dev) * c.inv_phi;
  if (ux) ux[o] = m.ux;
  if (uy) uy[o] = m.uy;
  if (THERMAL && Tout) Tout[o] = P.T0 + (gd[0] + gd[1] + gd[2] + gd[3] + gd[4]);
}

// one cell's (p, ux, uy, T) into out[0..3] (T = 0 without a temperature field)
template <int PREC, bool HET, bool THERMAL>
__global__ void k_probe(const StepParams P, int x, int y, float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float d[8], gd[5], ay;
  gather_state<PREC, HET, THERMAL>(P, P.src, P.gsrc, x, y, d, gd, ay);
  const Coef c = coef_at<HET>(P, x, y);
  const Macro m = macro_d2q8(d, c, P.ax, ay, P.rho0);
  out[0] = (P.p_rest + m.phip_dev) * c.inv_phi;
  out[1] = m.ux;
  out[2] = m.uy;
  out[3] = THERMAL ? P.T0 + (gd[0] + gd[1] + gd[2] + gd[3] + gd[4]) : 0.0f;
}

// --------------------------------------------------------------------------------------------
// FP64 reductions
// --------------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of two doubles; thread 0 receives the totals.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    a = l < nw ? sa[l] : 0.0;
    b = l < nw ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// Pass 1: per-block partial sums of |u(t) - u(t-1)|^2 and |u(t)|^2 into partial[2 * block];
// u(t-1) from the previous state (prev, gprev) or, if uprev is given, from its recorded
// components (dense [2][ny][nx]).
template <int PREC, bool HET, bool THERMAL>
__global__ void k_residual_partial(const StepParams P, const void* prev, const void* gprev, const float* __restrict__ uprev,
                                   double* __restrict__ partial) {
  double num = 0.0, den = 0.0;
  const int64_t n = (int64_t)P.nx * P.ny;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(k / P.nx), x = (int)(k - (int64_t)y * P.nx);
    const Coef c = coef_at<HET>(P, x, y);
    float d[8], gd[5], ay;
    gather_state<PREC, HET, THERMAL>(P, P.src, P.gsrc, x, y, d, gd, ay);
    const Macro a = macro_d2q8(d, c, P.ax, ay, P.rho0);
    double bx, by;
    if (uprev) {
      bx = uprev[k];
      by = uprev[n + k];
    } else {
      gather_state<PREC, HET, THERMAL>(P, prev, gprev, x, y, d, gd, ay);
      const Macro b = macro_d2q8(d, c, P.ax, ay, P.rho0);
      bx = b.ux;
      by = b.uy;
    }
    const double dx = (double)a.ux - bx, dy = (double)a.uy - by;
    num += dx * dx + dy * dy;
    den += (double)a.ux * a.ux + (double)a.uy * a.uy;
  }
  block_sum2(num, den);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = num;
    partial[2 * blockIdx.x + 1] = den;
  }
}

// Pass 2: one block adds the partials in a fixed order and writes out[0] = num, out[1] = den.
__global__ void k_sum_partials(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  double num = 0.0, den = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    num += partial[2 * i];
    den += partial[2 * i + 1];
  }
  block_sum2(num, den);
  if (threadIdx.x == 0) {
    out[0] = num;
    out[1] = den;
  }
}

// Nusselt number of the left (side 0) or right (side 1) wall: sum over rows of the outward
// normal temperature gradient at the wall, from the parabola through (wall, T_w), (1/2, T_a),
// (3/2, T_b): dT/ds = (9 T_a - T_b - 8 T_w) / 3.  out[0] = sum_y dT/ds.
template <int PREC>
__global__ void k_nusselt(const StepParams P, int side, double* __restrict__ out) {
  using T = typename Store<PREC>::T;
  const T* g = static_cast<const T*>(P.gsrc);
  double s = 0.0, unused = 0.0;
  const int xa = side == 0 ? 0 : P.nx - 1;
  const int xb = side == 0 ? 1 : P.nx - 2;
  if (P.bc_x == BC_NEE) {  // walls on the nodes x = 0, nx-1: dT/ds = (-3 T_0 + 4 T_1 - T_2) / 2
    const int xc = side == 0 ? 2 : P.nx - 3;
    const int y0 = P.bc_y == BC_NEE ? 1 : 0;  // corner rows belong to extrapolated bottom/top walls
    for (int y = y0 + (int)threadIdx.x; y < P.ny - y0; y += blockDim.x) {
      const double Ta = temperature_at<PREC>(P, g, xa, y), Tb = temperature_at<PREC>(P, g, xb, y);
      const double Tc = temperature_at<PREC>(P, g, xc, y);
      s += (-3.0 * Ta + 4.0 * Tb - Tc) / 2.0;
    }
    block_sum2(s, unused);
    if (threadIdx.x == 0) out[0] = s;
    return;
  }
  for (int y = threadIdx.x; y < P.ny; y += blockDim.x) {
    float ga[5], gb[5];
    pull_cell_g<PREC>(P, g, xa, y, ga);
    pull_cell_g<PREC>(P, g, xb, y, gb);
    const double Ta = (double)P.T0 + ((double)ga[0] + ga[1] + ga[2] + ga[3] + ga[4]);
    const double Tb = (double)P.T0 + ((double)gb[0] + gb[1] + gb[2] + gb[3] + gb[4]);
    s += (9.0 * Ta - Tb - 8.0 * (double)P.Tw[side]) / 3.0;
  }
  block_sum2(s, unused);
  if (threadIdx.x == 0) out[0] = s;
}

// --------------------------------------------------------------------------------------------
// host launchers
// --------------------------------------------------------------------------------------------
static dim3 row_grid(int n, int ny, int threads) { return dim3((n + threads - 1) / threads, ny); }

cudaError_t launch_medium(const float* eps, const float* K, float phi_u, float K_u, int nx, int ny, int pitch, float* phi_out,
                          float* K_out, unsigned int* err, int log_k, cudaStream_t s) {
  k_medium<<<row_grid(pitch, ny, 256), 256, 0, s>>>(eps, K, phi_u, K_u, nx, ny, pitch, phi_out, K_out, err, log_k);
  return cudaGetLastError();
}

#define LBM_DISPATCH_PH(prec, het, CALL)                    \
  do {                                                      \
    if (prec == PREC_FP32) {                                \
      if (het) { CALL(PREC_FP32, true); } else { CALL(PREC_FP32, false); } \
    } else if (prec == PREC_FP16) {                         \
      if (het) { CALL(PREC_FP16, true); } else { CALL(PREC_FP16, false); } \
    } else {                                                \
      if (het) { CALL(PREC_BF16, true); } else { CALL(PREC_BF16, false); } \
    }                                                       \
  } while (0)

#define LBM_DISPATCH_PHT(prec, het, thermal, CALL)                         \
  do {                                                                     \
    if (thermal) {                                                         \
      if (prec == PREC_FP32) { if (het) { CALL(PREC_FP32, true, true); } else { CALL(PREC_FP32, false, true); } } \
      else if (prec == PREC_FP16) { if (het) { CALL(PREC_FP16, true, true); } else { CALL(PREC_FP16, false, true); } } \
      else { if (het) { CALL(PREC_BF16, true, true); } else { CALL(PREC_BF16, false, true); } } \
    } else {                                                               \
      if (prec == PREC_FP32) { if (het) { CALL(PREC_FP32, true, false); } else { CALL(PREC_FP32, false, false); } } \
      else if (prec == PREC_FP16) { if (het) { CALL(PREC_FP16, true, false); } else { CALL(PREC_FP16, false, false); } } \
      else { if (het) { CALL(PREC_BF16, true, false); } else { CALL(PREC_BF16, false, false); } } \
    }                                                                      \
  } while (0)

cudaError_t launch_init(const StepParams& P, int prec, bool het, bool thermal, float p0, float ux0, float uy0, int phip_uniform,
                        float T_init, bool flow, bool temp, cudaStream_t s) {
  const dim3 grid = row_grid(P.pitch, P.ny, 128);
  if (flow) {
#define CALL_INIT(PR, H) k_init_flow<PR, H><<<grid, 128, 0, s>>>(P, p0, ux0, uy0, phip_uniform)
    LBM_DISPATCH_PH(prec, het, CALL_INIT);
#undef CALL_INIT
  }
  if (thermal && temp) {
    if (prec == PREC_FP32) k_init_thermal<PREC_FP32><<<grid, 128, 0, s>>>(P, T_init, ux0, uy0);
    else if (prec == PREC_FP16) k_init_thermal<PREC_FP16><<<grid, 128, 0, s>>>(P, T_init, ux0, uy0);
    else k_init_thermal<PREC_BF16><<<grid, 128, 0, s>>>(P, T_init, ux0, uy0);
  }
  return cudaGetLastError();
}

cudaError_t launch_import(const StepParams& P, int prec, const float* f, const float* g, cudaStream_t s) {
  const dim3 grid = row_grid(P.pitch, P.ny, 128);
  if (prec == PREC_FP32) k_import<PREC_FP32><<<grid, 128, 0, s>>>(P, f, g);
  else if (prec == PREC_FP16) k_import<PREC_FP16><<<grid, 128, 0, s>>>(P, f, g);
  else k_import<PREC_BF16><<<grid, 128, 0, s>>>(P, f, g);
  return cudaGetLastError();
}

cudaError_t launch_export(const StepParams& P, int prec, bool het, bool thermal, float* f, float* g, cudaStream_t s) {
  const dim3 grid = row_grid(P.nx, P.ny, 128);
#define CALL_EXP(PR, H, TH) k_export<PR, H, TH><<<grid, 128, 0, s>>>(P, f, g)
  LBM_DISPATCH_PHT(prec, het, thermal, CALL_EXP);
#undef CALL_EXP
  return cudaGetLastError();
}

cudaError_t launch_macros(const StepParams& P, int prec, bool het, bool thermal, float* p, float* ux, float* uy, float* T,
                          cudaStream_t s) {
  const dim3 grid = row_grid(P.nx, P.ny, 128);
#define CALL_MAC(PR, H, TH) k_macros<PR, H, TH><<<grid, 128, 0, s>>>(P, p, ux, uy, T)
  LBM_DISPATCH_PHT(prec, het, thermal, CALL_MAC);
#undef CALL_MAC
  return cudaGetLastError();
}

// a few floats, e.g. wall velocities from page-locked host memory that the device reads directly
__global__ void k_copy_small(float* __restrict__ dst, const float* __restrict__ src, int n) {
  const int i = threadIdx.x;
  if (i < n) dst[i] = src[i];
}

cudaError_t launch_copy_small(float* dst, const float* src, int n, cudaStream_t s) {
  k_copy_small<<<1, 32, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_probe(const StepParams& P, int prec, bool het, bool thermal, int x, int y, float* out, cudaStream_t s) {
#define CALL_PROBE(PR, H, TH) k_probe<PR, H, TH><<<1, 32, 0, s>>>(P, x, y, out)
  LBM_DISPATCH_PHT(prec, het, thermal, CALL_PROBE);
#undef CALL_PROBE
  return cudaGetLastError();
}

int residual_blocks(int nx, int ny) {
  const int64_t n = (int64_t)nx * ny;
  int64_t b = (n + 255) / 256;
  return (int)(b < kResidualMaxBlocks ? b : kResidualMaxBlocks);
}

cudaError_t launch_residual(const StepParams& P, int prec, bool het, bool thermal, const void* prev, const void* gprev,
                            const float* uprev, double* partial, int nblocks, double* out, cudaStream_t s) {
#define CALL_RES(PR, H, TH) k_residual_partial<PR, H, TH><<<nblocks, 256, 0, s>>>(P, prev, gprev, uprev, partial)
  LBM_DISPATCH_PHT(prec, het, thermal, CALL_RES);
#undef CALL_RES
  k_sum_partials<<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_nusselt(const StepParams& P, int prec, int side, double* out, cudaStream_t s) {
  if (prec == PREC_FP32) k_nusselt<PREC_FP32><<<1, 256, 0, s>>>(P, side, out);
  else if (prec == PREC_FP16) k_nusselt<PREC_FP16><<<1, 256, 0, s>>>(P, side, out);
  else k_nusselt<PREC_BF16><<<1, 256, 0, s>>>(P, side, out);
  return cudaGetLastError();
}

}  // namespace lbm
