// Fused stream-collide kernels of the porous D2Q8 MRT-LB method (Liu & He, arXiv 1311.7239,
// Eqs. 6-20) with the optional D2Q5 temperature equation (Appendix B) in the same pass.
//
// Layout and work split: planes [q][ny][pitch] with pitch a multiple of 128 elements; one CTA of
// 128 threads covers 512 consecutive cells of one row, each thread four consecutive cells.  The
// populations with e_x = 0 are read as aligned vectors; the six with e_x = +-1 are read as the
// same aligned vectors of the source row and shifted by one cell through a warp shuffle (the
// warp's first or last lane reads its one extra cell).  Cells on a wall row, on the first or
// last column, or next to a pressure column recompute their gathers with the generic edge rules.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStepThreads = 128;
constexpr int kCellsPerThread = 4;

// out[c] = row[x0 + c - SH] for c = 0..3 (SH = +1: pull from x-1, SH = -1: from x+1, 0: aligned)
template <int PREC, int SH>
__device__ __forceinline__ void gather4(const typename Store<PREC>::T* __restrict__ row, int xl, int pitch, int lane,
                                        float inv, float out[4]) {
  using S = Store<PREC>;
  float v[4];
  S::load4(row + xl, v, inv);
  if (SH == 0) {
    out[0] = v[0]; out[1] = v[1]; out[2] = v[2]; out[3] = v[3];
  } else if (SH == 1) {
    float left = __shfl_up_sync(kFull, v[3], 1);
    if (lane == 0) left = S::dec(row[xl > 0 ? xl - 1 : 0], inv);
    out[0] = left; out[1] = v[0]; out[2] = v[1]; out[3] = v[2];
  } else {
    float right = __shfl_down_sync(kFull, v[0], 1);
    if (lane == 31) right = S::dec(row[xl + 4 < pitch ? xl + 4 : pitch - 1], inv);
    out[0] = v[1]; out[1] = v[2]; out[2] = v[3]; out[3] = right;
  }
}

template <int PREC, bool HET, bool THERMAL>
__global__ void __launch_bounds__(kStepThreads) k_step(const StepParams P) {
  using S = Store<PREC>;
  using T = typename S::T;
  const T* __restrict__ src = static_cast<const T*>(P.src);
  T* __restrict__ dst = static_cast<T*>(P.dst);
  const int lane = threadIdx.x & 31;
  const int x0 = (blockIdx.x * kStepThreads + threadIdx.x) * kCellsPerThread;
  const int y = blockIdx.y;
  const int xl = x0 < P.pitch - 4 ? x0 : P.pitch - 4;  // loads stay inside the row
  int ym = y - 1, yp = y + 1;
  if (P.bc_y == BC_WALL) {
    ym = ym < 0 ? 0 : ym;  // wall rows are redone by the edge path
    yp = yp >= P.ny ? P.ny - 1 : yp;
  } else {
    ym = ym < 0 ? P.ny - 1 : ym;
    yp = yp >= P.ny ? 0 : yp;
  }
  const int64_t pl = P.plane;
  const int64_t rm = (int64_t)ym * P.pitch, r0 = (int64_t)y * P.pitch, rp = (int64_t)yp * P.pitch;
  const float inv = P.inv_scale;

  // pull streaming, Eq. 15: d_i(x) = d+_i(x - e_i)
  float d[8][4];
  gather4<PREC, 1>(src + 0 * pl + r0, xl, P.pitch, lane, inv, d[0]);   // e1 = ( 1, 0)
  gather4<PREC, 0>(src + 1 * pl + rm, xl, P.pitch, lane, inv, d[1]);   // e2 = ( 0, 1)
  gather4<PREC, -1>(src + 2 * pl + r0, xl, P.pitch, lane, inv, d[2]);  // e3 = (-1, 0)
  gather4<PREC, 0>(src + 3 * pl + rp, xl, P.pitch, lane, inv, d[3]);   // e4 = ( 0,-1)
  gather4<PREC, 1>(src + 4 * pl + rm, xl, P.pitch, lane, inv, d[4]);   // e5 = ( 1, 1)
  gather4<PREC, -1>(src + 5 * pl + rm, xl, P.pitch, lane, inv, d[5]);  // e6 = (-1, 1)
  gather4<PREC, -1>(src + 6 * pl + rp, xl, P.pitch, lane, inv, d[6]);  // e7 = (-1,-1)
  gather4<PREC, 1>(src + 7 * pl + rp, xl, P.pitch, lane, inv, d[7]);   // e8 = ( 1,-1)
  float g[5][4];
  const T* __restrict__ gsrc = static_cast<const T*>(P.gsrc);
  if (THERMAL) {
    gather4<PREC, 0>(gsrc + 0 * pl + r0, xl, P.pitch, lane, inv, g[0]);
    gather4<PREC, 1>(gsrc + 1 * pl + r0, xl, P.pitch, lane, inv, g[1]);
    gather4<PREC, 0>(gsrc + 2 * pl + rm, xl, P.pitch, lane, inv, g[2]);
    gather4<PREC, -1>(gsrc + 3 * pl + r0, xl, P.pitch, lane, inv, g[3]);
    gather4<PREC, 0>(gsrc + 4 * pl + rp, xl, P.pitch, lane, inv, g[4]);
  }
  if (x0 >= P.pitch) return;  // past the padded row: nothing to store (after the shuffles)

  const bool wall_row = P.bc_y == BC_WALL && (y == 0 || y == P.ny - 1);
  bool bad = false;
#pragma unroll
  for (int c = 0; c < kCellsPerThread; ++c) {
    const int x = x0 + c;
    float dc[8], gc[5];
#pragma unroll
    for (int i = 0; i < 8; ++i) dc[i] = d[i][c];
    if (THERMAL) {
#pragma unroll
      for (int i = 0; i < 5; ++i) gc[i] = g[i][c];
    }
    if (x < P.nx) {
      if (wall_row || x == 0 || x == P.nx - 1) {
        if (P.bc_x == BC_PRESSURE && (x == 0 || x == P.nx - 1))
          pressure_column<PREC, HET>(P, src, x, y, dc);
        else
          pull_cell<PREC>(P, src, x, y, dc);
        if (THERMAL) pull_cell_g<PREC>(P, gsrc, x, y, gc);
      }
      const Coef cf = coef_at<HET>(P, x, y);
      float ax = P.ax, ay = P.ay;
      if (THERMAL) {
        // buoyancy a = g beta (T - T0) j (Sec. 3.4), T = sum g of the pre-collision state
        const float dT = gc[0] + gc[1] + gc[2] + gc[3] + gc[4];
        ay += P.g_beta * dT;
      }
      float ux, uy, phip;
      collide_d2q8(dc, cf, ax, ay, P, ux, uy, phip);
      bad |= !(fabsf(ux) + fabsf(uy) < 1e30f);
      if (THERMAL) collide_d2q5(gc, ux, uy, P);
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) dc[i] = 0.0f;
      if (THERMAL) {
#pragma unroll
        for (int i = 0; i < 5; ++i) gc[i] = 0.0f;
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i][c] = dc[i];
    if (THERMAL) {
#pragma unroll
      for (int i = 0; i < 5; ++i) g[i][c] = gc[i];
    }
  }
  if (bad) atomicOr(P.err, 1u);
  const float sc = P.scale;
#pragma unroll
  for (int i = 0; i < 8; ++i) S::store4(dst + i * pl + r0 + x0, d[i], sc);
  if (THERMAL) {
    T* __restrict__ gdst = static_cast<T*>(P.gdst);
#pragma unroll
    for (int i = 0; i < 5; ++i) S::store4(gdst + i * pl + r0 + x0, g[i], sc);
  }
}

template <int PREC, bool HET, bool THERMAL>
static cudaError_t launch_step_t(const StepParams& P, cudaStream_t s) {
  const int per_block = kStepThreads * kCellsPerThread;
  dim3 grid((P.nx + per_block - 1) / per_block, P.ny);
  k_step<PREC, HET, THERMAL><<<grid, kStepThreads, 0, s>>>(P);
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_step_p(const StepParams& P, bool het, bool thermal, cudaStream_t s) {
  if (thermal) return het ? launch_step_t<PREC, true, true>(P, s) : launch_step_t<PREC, false, true>(P, s);
  return het ? launch_step_t<PREC, true, false>(P, s) : launch_step_t<PREC, false, false>(P, s);
}

cudaError_t launch_step(const StepParams& P, int prec, bool het, bool thermal, cudaStream_t s) {
  switch (prec) {
    case PREC_FP32: return launch_step_p<PREC_FP32>(P, het, thermal, s);
    case PREC_FP16: return launch_step_p<PREC_FP16>(P, het, thermal, s);
    default: return launch_step_p<PREC_BF16>(P, het, thermal, s);
  }
}

}  // namespace lbm
