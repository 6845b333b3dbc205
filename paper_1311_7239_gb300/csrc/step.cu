// Fused stream-collide kernel of the porous D2Q8 MRT-LB method (Liu & He, arXiv 1311.7239,
// Eqs. 6-20) with the optional D2Q5 temperature equation (Appendix B) in the same pass.
//
// Layout and work split: planes [q][ny][pitch] with pitch a multiple of 128 elements; a thread
// updates a group of four consecutive cells of one row, a CTA of 128 threads covers 512 cells.
// The populations with e_x = 0 are read as aligned vectors; the six with e_x = +-1 are read as
// the same aligned vectors of the source row and shifted by one cell through a warp shuffle (the
// warp's first or last lane reads its one extra cell).  The interior path has no boundary logic:
// the groups that touch a wall row or the first/last column (the "frame", a few cells per row)
// are done by the launch's first blocks with the generic boundary rules, and skipped by the rest.
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "tiles.cuh"

namespace lbm {

// Interior cells with 16-bit storage, where the step is bound by instruction issue rather than by
// HBM, are collided two at a time with the packed FP32 pairs (collide_pair): without temperature
// on any medium (step_item_words), with temperature on a uniform medium; FP32 storage keeps the
// scalar collision, whose lower register count holds more loads in flight.
template <int PREC, bool HET>
constexpr bool kPacked = PREC != PREC_FP32 && !HET;

template <int PREC, bool HET, bool THERMAL>
__device__ void frame_step(const StepParams& P, const Frame& F, int k) {
  using S = Store<PREC>;
  using T = typename S::T;
  int x, y;
  if (!frame_cell(F, P.ny, k, x, y)) return;
  if (!dbg_check(P, x >= 0 && x < P.pitch && y >= 0 && y < P.ny)) return;
  const int64_t o = (int64_t)y * P.pitch + x;
  T* dst = static_cast<T*>(P.dst);
  T* gdst = static_cast<T*>(P.gdst);
  float dc[8], gc[5];
  if (x < P.nx) {
    float ay = P.ay;
    if (THERMAL) {
      gather_cell_thermal<PREC, HET>(P, static_cast<const T*>(P.src), static_cast<const T*>(P.gsrc), x, y, dc, gc);
      ay += P.g_beta * (gc[0] + gc[1] + gc[2] + gc[3] + gc[4]);
    } else {
      gather_cell<PREC, HET>(P, static_cast<const T*>(P.src), x, y, dc);
    }
    const Coef cf = coef_at<HET>(P, x, y);
    float ux, uy, phip;
    collide_d2q8(dc, cf, P.ax, ay, P, ux, uy, phip);
    if (!(fabsf(ux) + fabsf(uy) < 1e30f)) atomicOr(P.err, 1u);
    if (THERMAL) collide_d2q5(gc, ux, uy, P);
  } else {  // row padding: zeros (never gathered by a lattice cell)
#pragma unroll
    for (int i = 0; i < 8; ++i) dc[i] = 0.0f;
#pragma unroll
    for (int i = 0; i < 5; ++i) gc[i] = 0.0f;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) dst[i * P.plane + o] = S::enc(dc[i], P.scale);
  if (THERMAL) {
#pragma unroll
    for (int i = 0; i < 5; ++i) gdst[i * P.plane + o] = S::enc(gc[i], P.scale);
  }
}

// Main item of the packed collision with 16-bit storage: the populations stay in their stored
// form (two cells per 32-bit word) until each pair is collided, which halves the registers that
// hold the gathered state.  A per-cell medium is read as float4 vectors of the four cells, issued
// ahead of the populations, and turned into pair coefficients per pair; with the temperature
// (uniform medium) the D2Q5 populations are gathered and collided the same way.
template <int PREC, bool HET, bool THERMAL, int NT>
__device__ __forceinline__ void step_item_words(const StepParams& P, const Tiling& tl, int item) {
  static_assert(!(HET && THERMAL), "the temperature step with a per-cell medium uses the scalar path");
  using S = Store<PREC>;
  using T = typename S::T;
  constexpr int C = kCellsPerThread;
  int x0, y;
  const bool has_group = main_group(tl, P.ny, NT, item - tl.frame_blocks, (int)threadIdx.x, x0, y);
  const T* __restrict__ src = static_cast<const T*>(P.src);
  const int lane = threadIdx.x & 31;
  int xl = x0 < P.pitch - C ? x0 : P.pitch - C;
  const bool idx_ok = dbg_check(P, y >= 0 && y < P.ny && xl >= 0);
  if (!idx_ok) y = xl = 0;  // (debug builds) keep the loads and shuffles inside the buffers
  int ym = y - 1, yp = y + 1;
  ym = ym < 0 ? P.ny - 1 : ym;
  yp = yp >= P.ny ? 0 : yp;
  const int64_t pl = P.plane;
  const int64_t rm = (int64_t)ym * P.pitch, r0 = (int64_t)y * P.pitch, rp = (int64_t)yp * P.pitch;
  float4 ph4, k4, sv4;
  if (HET) {
    ph4 = __ldg(reinterpret_cast<const float4*>(P.phi + r0 + xl));
    k4 = __ldg(reinterpret_cast<const float4*>(P.K + r0 + xl));
    sv4 = P.sv ? __ldg(reinterpret_cast<const float4*>(P.sv + r0 + xl)) : make_float4(P.s_v, P.s_v, P.s_v, P.s_v);
  }
  // pull streaming, Eq. 15, as stored (s d): w[i] = pairs (c0, c1), (c2, c3) of population i
  uint32_t w[8][2];
  gather4w<PREC, 1>(src + 0 * pl + r0, xl, P.pitch, lane, w[0]);   // e1 = ( 1, 0)
  gather4w<PREC, 0>(src + 1 * pl + rm, xl, P.pitch, lane, w[1]);   // e2 = ( 0, 1)
  gather4w<PREC, -1>(src + 2 * pl + r0, xl, P.pitch, lane, w[2]);  // e3 = (-1, 0)
  gather4w<PREC, 0>(src + 3 * pl + rp, xl, P.pitch, lane, w[3]);   // e4 = ( 0,-1)
  gather4w<PREC, 1>(src + 4 * pl + rm, xl, P.pitch, lane, w[4]);   // e5 = ( 1, 1)
  gather4w<PREC, -1>(src + 5 * pl + rm, xl, P.pitch, lane, w[5]);  // e6 = (-1, 1)
  gather4w<PREC, -1>(src + 6 * pl + rp, xl, P.pitch, lane, w[6]);  // e7 = (-1,-1)
  gather4w<PREC, 1>(src + 7 * pl + rp, xl, P.pitch, lane, w[7]);   // e8 = ( 1,-1)
  uint32_t gw[5][2];
  if (THERMAL) {  // Eq. B.2: g_i(x) = g+_i(x - e_i), D2Q5 (rest, e1..e4)
    const T* __restrict__ gsrc = static_cast<const T*>(P.gsrc);
    gather4w<PREC, 0>(gsrc + 0 * pl + r0, xl, P.pitch, lane, gw[0]);
    gather4w<PREC, 1>(gsrc + 1 * pl + r0, xl, P.pitch, lane, gw[1]);
    gather4w<PREC, 0>(gsrc + 2 * pl + rm, xl, P.pitch, lane, gw[2]);
    gather4w<PREC, -1>(gsrc + 3 * pl + r0, xl, P.pitch, lane, gw[3]);
    gather4w<PREC, 0>(gsrc + 4 * pl + rp, xl, P.pitch, lane, gw[4]);
  }
  const bool wall_row = (P.bc_y == BC_WALL || P.bc_y == BC_NEE) && (y == 0 || y == P.ny - 1);
  if (!has_group || !idx_ok || wall_row || x0 == 0 || x0 + C >= P.nx) return;
  float check = 0.0f;
#pragma unroll
  for (int h = 0; h < C / 2; ++h) {
    float2 dp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) dp[i] = S::w2f(w[i][h]);
    float2 ux, uy;
    if (HET) {
      float2 hx, hy;
      const PairCoef c = pair_coef_het(P, h ? make_float2(ph4.z, ph4.w) : make_float2(ph4.x, ph4.y),
                                       h ? make_float2(k4.z, k4.w) : make_float2(k4.x, k4.y),
                                       h ? make_float2(sv4.z, sv4.w) : make_float2(sv4.x, sv4.y), hx, hy);
      collide_pair(dp, c, hx, hy, P.pc, ux, uy);
    } else if (THERMAL) {
      float2 gp[5];
#pragma unroll
      for (int i = 0; i < 5; ++i) gp[i] = S::w2f(gw[i][h]);
      // a = g beta (T - T0) j added to the body force (Boussinesq): phi a_y / 2 of the two cells
      const float2 sTd = add2(add2(add2(gp[0], gp[1]), add2(gp[2], gp[3])), gp[4]);  // s (T - T0)
      const float2 hy = mul2(f2(P.phi_u), fma2(f2(0.5f * P.g_beta * P.inv_scale), sTd, f2(P.pc.hay)));
      collide_pair(dp, pair_coef_uniform(P.pc), f2(P.pc.u_hx), hy, P.pc, ux, uy);
      collide_d2q5_pair(gp, ux, uy, P);
#pragma unroll
      for (int i = 0; i < 5; ++i) gw[i][h] = S::f2w(gp[i]);
    } else {
      collide_pair(dp, pair_coef_uniform(P.pc), f2(P.pc.u_hx), f2(P.pc.u_hy), P.pc, ux, uy);
    }
    check += (fabsf(ux.x) + fabsf(uy.x)) + (fabsf(ux.y) + fabsf(uy.y));
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i][h] = S::f2w(dp[i]);
  }
  if (!(check < 1e30f)) atomicOr(P.err, 1u);  // non-finite velocity in these cells
  T* __restrict__ dst = static_cast<T*>(P.dst);
#pragma unroll
  for (int i = 0; i < 8; ++i) *reinterpret_cast<uint2*>(dst + i * pl + r0 + x0) = make_uint2(w[i][0], w[i][1]);
  if (THERMAL) {
    T* __restrict__ gdst = static_cast<T*>(P.gdst);
#pragma unroll
    for (int i = 0; i < 5; ++i) *reinterpret_cast<uint2*>(gdst + i * pl + r0 + x0) = make_uint2(gw[i][0], gw[i][1]);
  }
}

// Work item `item` of one lattice, for CTAs of NT threads: items [0, frame_blocks) do the frame,
// the rest cover the lattice row by row, gx items per row, and store every group that is not a
// frame group.  Every thread of the CTA calls this with the same item (warp shuffles inside).
template <int PREC, bool HET, bool THERMAL, int NT>
__device__ __forceinline__ void step_item(const StepParams& P, const Tiling& tl, int item) {
  using S = Store<PREC>;
  using T = typename S::T;
  constexpr int C = kCellsPerThread;
  if (item < tl.frame_blocks) {
    const Frame F = frame_of(P.nx, P.ny, P.bc_y, C);
    frame_step<PREC, HET, THERMAL>(P, F, item * NT + (int)threadIdx.x);
    return;
  }
  if constexpr (PREC != PREC_FP32 && !(HET && THERMAL)) {
    step_item_words<PREC, HET, THERMAL, NT>(P, tl, item);
    return;
  }
  int x0, y;
  const bool has_group = main_group(tl, P.ny, NT, item - tl.frame_blocks, (int)threadIdx.x, x0, y);
  const T* __restrict__ src = static_cast<const T*>(P.src);
  T* __restrict__ dst = static_cast<T*>(P.dst);
  const int lane = threadIdx.x & 31;
  int xl = x0 < P.pitch - C ? x0 : P.pitch - C;  // loads stay inside the row
  const bool idx_ok = dbg_check(P, y >= 0 && y < P.ny && xl >= 0);
  if (!idx_ok) y = xl = 0;  // (debug builds) keep the loads and shuffles inside the buffers
  // source rows of e_y = +1 and -1 (periodic wrap; wall rows belong to the frame)
  int ym = y - 1, yp = y + 1;
  ym = ym < 0 ? P.ny - 1 : ym;
  yp = yp >= P.ny ? 0 : yp;
  const int64_t pl = P.plane;
  const int64_t rm = (int64_t)ym * P.pitch, r0 = (int64_t)y * P.pitch, rp = (int64_t)yp * P.pitch;
  const float inv = P.inv_scale;
  // medium of the four cells, issued ahead of the populations (aligned: x0 and the pitch are
  // multiples of 4 and the fields are allocated like the populations)
  float4 ph4, k4;
  if (HET) {
    ph4 = __ldg(reinterpret_cast<const float4*>(P.phi + r0 + xl));
    k4 = __ldg(reinterpret_cast<const float4*>(P.K + r0 + xl));
  }

  // pull streaming, Eq. 15: d_i(x) = d+_i(x - e_i) (as stored, s d, for the pair collision)
  constexpr bool R = kPacked<PREC, HET>;
  float d[8][C];
  gather4<PREC, 1, R>(src + 0 * pl + r0, xl, P.pitch, lane, inv, d[0]);   // e1 = ( 1, 0)
  gather4<PREC, 0, R>(src + 1 * pl + rm, xl, P.pitch, lane, inv, d[1]);   // e2 = ( 0, 1)
  gather4<PREC, -1, R>(src + 2 * pl + r0, xl, P.pitch, lane, inv, d[2]);  // e3 = (-1, 0)
  gather4<PREC, 0, R>(src + 3 * pl + rp, xl, P.pitch, lane, inv, d[3]);   // e4 = ( 0,-1)
  gather4<PREC, 1, R>(src + 4 * pl + rm, xl, P.pitch, lane, inv, d[4]);   // e5 = ( 1, 1)
  gather4<PREC, -1, R>(src + 5 * pl + rm, xl, P.pitch, lane, inv, d[5]);  // e6 = (-1, 1)
  gather4<PREC, -1, R>(src + 6 * pl + rp, xl, P.pitch, lane, inv, d[6]);  // e7 = (-1,-1)
  gather4<PREC, 1, R>(src + 7 * pl + rp, xl, P.pitch, lane, inv, d[7]);   // e8 = ( 1,-1)
  float g[5][C];
  if (THERMAL) {
    const T* __restrict__ gsrc = static_cast<const T*>(P.gsrc);
    gather4<PREC, 0>(gsrc + 0 * pl + r0, xl, P.pitch, lane, inv, g[0]);
    gather4<PREC, 1>(gsrc + 1 * pl + r0, xl, P.pitch, lane, inv, g[1]);
    gather4<PREC, 0>(gsrc + 2 * pl + rm, xl, P.pitch, lane, inv, g[2]);
    gather4<PREC, -1>(gsrc + 3 * pl + r0, xl, P.pitch, lane, inv, g[3]);
    gather4<PREC, 0>(gsrc + 4 * pl + rp, xl, P.pitch, lane, inv, g[4]);
  }
  // (after the shuffles) frame groups and groups past the row are not stored here
  const bool wall_row = (P.bc_y == BC_WALL || P.bc_y == BC_NEE) && (y == 0 || y == P.ny - 1);
  if (!has_group || !idx_ok || wall_row || x0 == 0 || x0 + C >= P.nx) return;

  float check = 0.0f;
  if constexpr (R) {
#pragma unroll
    for (int h = 0; h < C / 2; ++h) {  // cells (x0 + 2h, x0 + 2h + 1) as one packed pair
      const int c0 = 2 * h, c1 = 2 * h + 1;
      float2 dp[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) dp[i] = make_float2(d[i][c0], d[i][c1]);
      float2 hy = f2(P.pc.u_hy);
      if (THERMAL) {  // a_y = g beta (T - T0) j added to the body force (Boussinesq)
        const float2 Td = make_float2(g[0][c0] + g[1][c0] + g[2][c0] + g[3][c0] + g[4][c0],
                                      g[0][c1] + g[1][c1] + g[2][c1] + g[3][c1] + g[4][c1]);
        hy = mul2(f2(P.phi_u), fma2(f2(0.5f * P.g_beta), Td, f2(P.pc.hay)));
      }
      float2 ux, uy;
      collide_pair(dp, pair_coef_uniform(P.pc), f2(P.pc.u_hx), hy, P.pc, ux, uy);
      check += (fabsf(ux.x) + fabsf(uy.x)) + (fabsf(ux.y) + fabsf(uy.y));
#pragma unroll
      for (int i = 0; i < 8; ++i) S::store2r(dst + i * pl + r0 + x0 + c0, dp[i]);
      if (THERMAL) {
        float gc[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) gc[i] = g[i][c0];
        collide_d2q5(gc, ux.x, uy.x, P);
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i][c0] = gc[i];
#pragma unroll
        for (int i = 0; i < 5; ++i) gc[i] = g[i][c1];
        collide_d2q5(gc, ux.y, uy.y, P);
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i][c1] = gc[i];
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float dc[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) dc[i] = d[i][c];
      const Coef cf = HET ? coef_of(P, f4_get(ph4, c), f4_get(k4, c), P.sv ? __ldg(P.sv + r0 + x0 + c) : P.s_v) : coef_uniform(P);
      float ay = P.ay;
      if (THERMAL) ay += P.g_beta * (g[0][c] + g[1][c] + g[2][c] + g[3][c] + g[4][c]);  // a = g beta (T - T0) j
      float ux, uy, phip;
      collide_d2q8(dc, cf, P.ax, ay, P, ux, uy, phip);
      check += fabsf(ux) + fabsf(uy);
#pragma unroll
      for (int i = 0; i < 8; ++i) d[i][c] = dc[i];
      if (THERMAL) {
        float gc[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) gc[i] = g[i][c];
        collide_d2q5(gc, ux, uy, P);
#pragma unroll
        for (int i = 0; i < 5; ++i) g[i][c] = gc[i];
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) S::store4(dst + i * pl + r0 + x0, d[i], P.scale);
  }
  if (!(check < 1e30f)) atomicOr(P.err, 1u);  // non-finite velocity in these cells
  const float sc = P.scale;
  if (THERMAL) {
    T* __restrict__ gdst = static_cast<T*>(P.gdst);
#pragma unroll
    for (int i = 0; i < 5; ++i) S::store4(gdst + i * pl + r0 + x0, g[i], sc);
  }
}

// One time step of one lattice: one CTA per work item (flat tiling).  Register caps (measured): 8
// CTAs (32 warps) per SM for the flow alone (64 registers), with every storage precision; 6 with
// the temperature populations (80 registers; the 16-bit uniform-medium form runs 8 % faster than
// at 96), 5 (96) for the scalar 16-bit temperature step of a per-cell medium.
template <int PREC, bool HET, bool THERMAL>
__global__ void __launch_bounds__(kStepThreads, THERMAL ? (PREC != PREC_FP32 && HET ? 5 : 6) : 8) k_step(const StepParams P, Tiling tl) {
  step_item<PREC, HET, THERMAL, kStepThreads>(P, tl, blockIdx.x);
}

template <int PREC, bool HET, bool THERMAL>
static cudaError_t launch_step_t(const StepParams& P, cudaStream_t s) {
  const Tiling tl = tiling_of(P.nx, P.ny, P.bc_y, kStepThreads, true);
  const long long blocks = (long long)tl.frame_blocks + main_items(tl, P.ny, kStepThreads);
  k_step<PREC, HET, THERMAL><<<(unsigned)blocks, kStepThreads, 0, s>>>(P, tl);
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_step_p(const StepParams& P, bool het, bool thermal, cudaStream_t s) {
  if (thermal) return het ? launch_step_t<PREC, true, true>(P, s) : launch_step_t<PREC, false, true>(P, s);
  return het ? launch_step_t<PREC, true, false>(P, s) : launch_step_t<PREC, false, false>(P, s);
}

// --------------------------------------------------------------------------------------------
cudaError_t launch_step(const StepParams& P, int prec, bool het, bool thermal, cudaStream_t s) {
  switch (prec) {
    case PREC_FP32: return launch_step_p<PREC_FP32>(P, het, thermal, s);
    case PREC_FP16: return launch_step_p<PREC_FP16>(P, het, thermal, s);
    default: return launch_step_p<PREC_BF16>(P, het, thermal, s);
  }
}

// --------------------------------------------------------------------------------------------
// Batched ensemble: one launch advances every lattice of a batch by one step.  The work items of
// the lattices are concatenated (item_start, ascending); lattice d's parameters for the current
// buffer parity are Pd[d], copied once per CTA into shared memory (the streamed populations would
// otherwise evict them from L1 between items).  Two launch forms:
//   k_step_batch_items  one CTA per work item; item_lattice[item] names the item's lattice;
//   k_step_batch        persistent: CTA b walks the contiguous range [b * chunk, (b + 1) * chunk)
//                       of items, looks its lattice up once (binary search) and moves on to the
//                       next lattice only when the range crosses into it.
// --------------------------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void load_params(StepParams& sP, const StepParams* __restrict__ Pd, int d) {
  static_assert(sizeof(StepParams) % 8 == 0, "parameters are copied as 8-byte words");
  const unsigned long long* from = reinterpret_cast<const unsigned long long*>(Pd + d);
  unsigned long long* to = reinterpret_cast<unsigned long long*>(&sP);
  for (int i = threadIdx.x; i < (int)(sizeof(StepParams) / 8); i += NT) to[i] = from[i];
}

// Register caps (measured on a 512-lattice ensemble): the streaming rate follows the number of
// resident warps, so the per-item form is held to 64 registers with FP32 storage (32 warps per SM,
// a few bytes of spill) and to 80 with 16-bit storage (24 warps; its packed collision spills
// 200 bytes at 64 and runs 13 % slower), the persistent form to 85 (24 warps); uncapped they take
// 72-108 registers and run 1.2-1.5x slower.  flat: the lattices' tiling (tiling_of).
template <int PREC, int NT>
__global__ void __launch_bounds__(NT, (PREC == PREC_FP32 ? 1024 : 768) / NT) k_step_batch_items(const StepParams* __restrict__ Pd,
                                                                                         const int64_t* __restrict__ item_start,
                                                                                         const int* __restrict__ item_lattice, int flat) {
  __shared__ StepParams sP;
  const int d = item_lattice[blockIdx.x];
  load_params<NT>(sP, Pd, d);
  __syncthreads();
  const Tiling tl = tiling_of(sP.nx, sP.ny, sP.bc_y, NT, flat != 0);
  step_item<PREC, true, false, NT>(sP, tl, (int)((int64_t)blockIdx.x - item_start[d]));
}

// The per-item form when the lattices share rho0, s_e, s_q and the storage scale: U (one lattice's
// parameters, by value: the kernel's constant bank) supplies those and the collision constants, the
// record of the item's lattice the fields that differ, so a main item starts its gathers without
// staging the parameter set in shared memory and keeps the constants out of the registers.  Frame
// items, which use every parameter, stage the lattice's set as the general form.  Register caps
// (512-lattice ensemble): FP16 at 72 registers 122.1 GLUPS (117.7 at 64, 112.9 at 80; the staged
// form 102.4), BF16 and FP32 at 64 (BF16 113.4-114.7 at 64-80).
template <int PREC, int NT>
__global__ void __launch_bounds__(NT, (PREC == PREC_FP16 ? 896 : 1024) / NT)
    k_step_batch_items_shared(const StepParams U, const BatchRec* __restrict__ R, const StepParams* __restrict__ Pd,
                              const int64_t* __restrict__ item_start, const int* __restrict__ item_lattice, int flat) {
  const int d = item_lattice[blockIdx.x];
  const BatchRec& r = R[d];
  const Tiling tl = tiling_of(r.nx, r.ny, r.bc_y, NT, flat != 0);
  const int item = (int)((int64_t)blockIdx.x - item_start[d]);
  if (item < tl.frame_blocks) {
    __shared__ StepParams sP;
    load_params<NT>(sP, Pd, d);
    __syncthreads();
    step_item<PREC, true, false, NT>(sP, tl, item);
    return;
  }
  StepParams Q = U;
  Q.src = r.src;
  Q.dst = r.dst;
  Q.phi = r.phi;
  Q.K = r.K;
  Q.sv = nullptr;
  Q.uw = r.uw;
  Q.plane = r.plane;
  Q.nx = r.nx;
  Q.ny = r.ny;
  Q.pitch = r.pitch;
  Q.bc_x = r.bc_x;
  Q.bc_y = r.bc_y;
  Q.forch = r.forch;
  Q.nu = r.nu;
  Q.s_v = r.s_v;
  Q.ax = r.ax;
  Q.ay = r.ay;
  Q.pc.hax = 0.5f * r.ax;
  Q.pc.hay = 0.5f * r.ay;
  if constexpr (PREC == PREC_FP32) step_item<PREC, true, false, NT>(Q, tl, item);
  else step_item_words<PREC, true, false, NT>(Q, tl, item);
}

template <int PREC, int NT>
__global__ void __launch_bounds__(NT, 768 / NT) k_step_batch(const StepParams* __restrict__ Pd, const int64_t* __restrict__ item_start, int n,
                                                   int64_t total, int flat) {
  __shared__ StepParams sP;
  const int64_t chunk = (total + gridDim.x - 1) / gridDim.x;
  const int64_t begin = (int64_t)blockIdx.x * chunk;
  const int64_t end = begin + chunk < total ? begin + chunk : total;
  if (begin >= end) return;
  int lo = 0, hi = n - 1;  // last d with item_start[d] <= begin
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (item_start[mid] <= begin) lo = mid; else hi = mid - 1;
  }
  int64_t first = item_start[lo];
  int64_t next = lo + 1 < n ? item_start[lo + 1] : total;
  load_params<NT>(sP, Pd, lo);
  __syncthreads();
  Tiling tl = tiling_of(sP.nx, sP.ny, sP.bc_y, NT, flat != 0);
  for (int64_t it = begin; it < end; ++it) {
    if (it >= next) {  // the range crosses into the next lattice(s): uniform over the CTA
      while (it >= next) {
        ++lo;
        next = lo + 1 < n ? item_start[lo + 1] : total;
      }
      first = item_start[lo];
      __syncthreads();  // every thread is done with the previous parameters
      load_params<NT>(sP, Pd, lo);
      __syncthreads();
      tl = tiling_of(sP.nx, sP.ny, sP.bc_y, NT, flat != 0);
    }
    step_item<PREC, true, false, NT>(sP, tl, (int)(it - first));
  }
}

}  // namespace lbm

namespace lbm {

int64_t batch_items(int nx, int ny, int bc_y, int nt, int flat) {
  const Tiling tl = tiling_of(nx, ny, bc_y, nt, flat != 0);
  return (int64_t)tl.frame_blocks + main_items(tl, ny, nt);
}

template <int PREC, int NT>
static void launch_batch_t(const StepParams* Pd, const int64_t* item_start, const int* item_lattice, int n, int64_t total, int grid,
                           int flat, cudaStream_t s) {
  if (item_lattice)
    k_step_batch_items<PREC, NT><<<(unsigned)total, NT, 0, s>>>(Pd, item_start, item_lattice, flat);
  else
    k_step_batch<PREC, NT><<<grid, NT, 0, s>>>(Pd, item_start, n, total, flat);
}

template <int PREC>
static cudaError_t launch_batch_p(const StepParams* Pd, const int64_t* item_start, const int* item_lattice, int n, int64_t total,
                                  int nt, int grid, int flat, cudaStream_t s) {
  switch (nt) {
    case 64: launch_batch_t<PREC, 64>(Pd, item_start, item_lattice, n, total, grid, flat, s); break;
    case 256: launch_batch_t<PREC, 256>(Pd, item_start, item_lattice, n, total, grid, flat, s); break;
    default: launch_batch_t<PREC, 128>(Pd, item_start, item_lattice, n, total, grid, flat, s); break;
  }
  return cudaGetLastError();
}

template <int PREC>
static void launch_shared_p(const StepParams& U, const BatchRec* R, const StepParams* Pd, const int64_t* item_start,
                            const int* item_lattice, int64_t total, int nt, int flat, cudaStream_t s) {
  switch (nt) {
    case 64: k_step_batch_items_shared<PREC, 64><<<(unsigned)total, 64, 0, s>>>(U, R, Pd, item_start, item_lattice, flat); break;
    case 256: k_step_batch_items_shared<PREC, 256><<<(unsigned)total, 256, 0, s>>>(U, R, Pd, item_start, item_lattice, flat); break;
    default: k_step_batch_items_shared<PREC, 128><<<(unsigned)total, 128, 0, s>>>(U, R, Pd, item_start, item_lattice, flat); break;
  }
}

cudaError_t launch_step_batch_shared(const StepParams& U, const BatchRec* R, const StepParams* Pd, const int64_t* item_start,
                                     const int* item_lattice, int64_t total, int prec, int nt, int flat, cudaStream_t s) {
  if (prec == PREC_FP16) launch_shared_p<PREC_FP16>(U, R, Pd, item_start, item_lattice, total, nt, flat, s);
  else if (prec == PREC_BF16) launch_shared_p<PREC_BF16>(U, R, Pd, item_start, item_lattice, total, nt, flat, s);
  else launch_shared_p<PREC_FP32>(U, R, Pd, item_start, item_lattice, total, nt, flat, s);
  return cudaGetLastError();
}

// Largest number of CTAs of the persistent batched kernel (prec, nt) resident on one SM.
int batch_max_ctas_per_sm(int prec, int nt) {
  int k = 0;
  const void* fn = nullptr;
#define LBM_BATCH_FN(PR)                                                      \
  (nt == 64 ? (const void*)k_step_batch<PR, 64> : nt == 256 ? (const void*)k_step_batch<PR, 256> \
                                                            : (const void*)k_step_batch<PR, 128>)
  fn = prec == PREC_FP32 ? LBM_BATCH_FN(PREC_FP32) : prec == PREC_FP16 ? LBM_BATCH_FN(PREC_FP16) : LBM_BATCH_FN(PREC_BF16);
#undef LBM_BATCH_FN
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, fn, nt, 0) != cudaSuccess) return 1;
  return k > 0 ? k : 1;
}

cudaError_t launch_step_batch(const StepParams* Pd, const int64_t* item_start, const int* item_lattice, int n, int64_t total, int prec,
                              int nt, int grid, int flat, cudaStream_t s) {
  if (prec == PREC_FP32) return launch_batch_p<PREC_FP32>(Pd, item_start, item_lattice, n, total, nt, grid, flat, s);
  if (prec == PREC_FP16) return launch_batch_p<PREC_FP16>(Pd, item_start, item_lattice, n, total, nt, grid, flat, s);
  return launch_batch_p<PREC_BF16>(Pd, item_start, item_lattice, n, total, nt, grid, flat, s);
}

}  // namespace lbm
