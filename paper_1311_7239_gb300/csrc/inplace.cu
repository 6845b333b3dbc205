// In-place ("esoteric pull") form of the fused stream-collide step: one population buffer instead
// of the two of the A-B form, with the same arithmetic per cell (Eqs. 6-20, and Eq. B.2 for the
// temperature).  The slot rules are those of ip_off in lbm_device.cuh: at parity PAR a cell reads
// population i from plane (PAR ? i : opp(i)), at the cell itself for the positive member of each
// opposite pair (e1, e2, e5, e8) and at c - e_i for the others, and writes its post-collision
// population opp(i) back into the slot it read i from.  Per step and cell the traffic is that of
// the A-B form (8 loads, 8 stores); the footprint of the populations halves.
//
// Work split: a thread updates four consecutive cells of one row.  Of the slots it touches, five
// are the aligned four-cell vectors of rows y and y + 1 (positive members and e4 = (0, -1)); the
// three with e_x = -1 sit one cell to the right (x0 + 1 .. x0 + 4) and are moved as one cell, an
// aligned pair and one cell, so that a thread touches no slot of another thread's cells.  The
// groups with a cell on a wall or on the last column (where the right neighbour wraps or is a
// ghost slot) form a "frame" that the launch's first blocks do cell by cell with the generic
// rules, so that the warps of the interior never diverge.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

constexpr int kIpThreads = 128;
constexpr int kIpCells = 4;

// u of the collision at (x, y) into the record of the previous state's velocity (the residual's
// u(t-1) once the step is done)
__device__ __forceinline__ void record_u(const StepParams& P, int x, int y, float ux, float uy) {
  const int64_t o = (int64_t)y * P.nx + x;
  P.urec[o] = ux;
  P.urec[(int64_t)P.nx * P.ny + o] = uy;
}

// the same for the two cells x, x + 1 (x even): one 8-byte store per component when the record's
// rows start on 8 bytes (nx even)
__device__ __forceinline__ void record_u2(const StepParams& P, int x, int y, float2 ux, float2 uy) {
  const int64_t o = (int64_t)y * P.nx + x, n = (int64_t)P.nx * P.ny;
  if ((P.nx & 1) == 0) {
    *reinterpret_cast<float2*>(P.urec + o) = ux;
    *reinterpret_cast<float2*>(P.urec + n + o) = uy;
  } else {
    P.urec[o] = ux.x;
    P.urec[o + 1] = ux.y;
    P.urec[n + o] = uy.x;
    P.urec[n + o + 1] = uy.y;
  }
}

// Extrapolated sides (wall nodes and pressure columns): a boundary node's pre-collision state is
// a function of its inner neighbour's, which that neighbour's own update overwrites in the same
// pass.  So k_edge_ip computes the states of all boundary nodes of the coming step first (the
// rules of gather_cell / gather_cell_thermal on the unchanged buffer) into FP32 planes
// [8 (+5)][2 (nx + ny)], and the step reads them from there; the node's own slots are written as
// any cell's.  Plane index of a boundary node: bottom row x, top row nx + x, left column (rows
// 1..ny-2) 2 nx + y, right column 2 nx + ny + y.
__device__ __forceinline__ int edge_index(const StepParams& P, int x, int y) {
  if (y == 0) return x;
  if (y == P.ny - 1) return P.nx + x;
  return 2 * P.nx + (x == 0 ? y : P.ny + y);
}

__device__ __forceinline__ bool boundary_node(const StepParams& P, int x, int y) {
  int xn, yn, w;
  return nee_node(P, x, y, xn, yn, w) || (P.bc_x == BC_PRESSURE && (x == 0 || x == P.nx - 1));
}

// Eight lanes per boundary node, lane i pulling population i (and temperature population i < 5) of
// the node's inner neighbour, so that the scattered loads of a node are in flight together; the
// pulled state is then shared within the lane group and every lane applies the node's rule to the
// whole state (the functions gather_cell uses, so the result is bitwise that of the A-B form) and
// stores its own population.
template <int PREC, bool HET, bool THERMAL>
__global__ void k_edge_ip(const StepParams P) {
  using T = typename Store<PREC>::T;
  const int n = 2 * (P.nx + P.ny);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = t >> 3, lane = t & 7;
  if (k >= n) return;  // whole lane groups leave together (as below: x, y and the rule depend on k only)
  int x, y;
  if (k < 2 * P.nx) {
    if (k >= P.nx && P.ny == 1) return;  // one row: the bottom range has it
    y = k < P.nx ? 0 : P.ny - 1;
    x = k < P.nx ? k : k - P.nx;
  } else {
    const int r = k - 2 * P.nx;
    x = r < P.ny ? 0 : P.nx - 1;
    y = r < P.ny ? r : r - P.ny;
    if (y == 0 || y == P.ny - 1) return;  // the rows' ranges have the corners
  }
  int xn, yn, w;
  const bool wall = nee_node(P, x, y, xn, yn, w);
  if (!wall) {
    if (!(P.bc_x == BC_PRESSURE && (x == 0 || x == P.nx - 1))) return;
    xn = x == 0 ? 1 : P.nx - 2;
    yn = y;
  }
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  const int base = threadIdx.x & 24;
  const float zi = pull_one<PREC>(P, static_cast<const T*>(P.src), xn, yn, lane);
  // temperature: a wall node extrapolates from nb, a pressure column keeps its own pulled state
  const float gi = (THERMAL && lane < 5) ? pull_one_g<PREC>(P, static_cast<const T*>(P.gsrc), wall ? xn : x, wall ? yn : y, lane) : 0.0f;
  float dn[8], gn[5], d[8], g[5];
#pragma unroll
  for (int j = 0; j < 8; ++j) dn[j] = __shfl_sync(gm, zi, base + j);
  if (THERMAL) {
#pragma unroll
    for (int j = 0; j < 5; ++j) gn[j] = __shfl_sync(gm, gi, base + j);
  }
  if (wall) {
    if (THERMAL) {
      thermal_wall_node_from<HET>(P, dn, gn, x, y, xn, yn, w, d, g);
    } else {
      float ux, uy;
      wall_node_from<HET>(P, dn, x, y, xn, yn, w, P.ay, d, ux, uy);
    }
  } else {
    pressure_column_from<HET>(P, dn, x, y, d);
    if (THERMAL) {
#pragma unroll
      for (int j = 0; j < 5; ++j) g[j] = gn[j];
    }
  }
  float dv = d[0], gv = THERMAL ? g[0] : 0.0f;
#pragma unroll
  for (int j = 1; j < 8; ++j) dv = lane == j ? d[j] : dv;
  if (THERMAL) {
#pragma unroll
    for (int j = 1; j < 5; ++j) gv = lane == j ? g[j] : gv;
  }
  P.edge[lane * n + k] = dv;
  if (THERMAL && lane < 5) P.edge[(8 + lane) * n + k] = gv;
}

// one cell with the generic slot rules: pulls with bounce-back (or, for a boundary node of an
// extrapolated side, the state k_edge_ip computed), collision, stores into the slots of the next
// parity (ghost slots for populations that leave through a wall)
template <int PREC, bool HET, bool THERMAL, bool REC>
__device__ __noinline__ void ip_cell(const StepParams& P, typename Store<PREC>::T* A, typename Store<PREC>::T* G, int x, int y) {
  using S = Store<PREC>;
  float d[8], g[5];
  if (P.edge && boundary_node(P, x, y)) {
    const int n = 2 * (P.nx + P.ny), e = edge_index(P, x, y);
#pragma unroll
    for (int i = 0; i < 8; ++i) d[i] = P.edge[i * n + e];
    if (THERMAL) {
#pragma unroll
      for (int i = 0; i < 5; ++i) g[i] = P.edge[(8 + i) * n + e];
    }
  } else {
    pull_cell<PREC>(P, A, x, y, d);
    if (THERMAL) pull_cell_g<PREC>(P, G, x, y, g);
  }
  float ay = P.ay;
  if (THERMAL) ay += P.g_beta * (g[0] + g[1] + g[2] + g[3] + g[4]);  // a = g beta (T - T0) j
  const Coef cf = coef_at<HET>(P, x, y);
  float ux, uy, phip;
  collide_d2q8(d, cf, P.ax, ay, P, ux, uy, phip);
  if (!(fabsf(ux) + fabsf(uy) < 1e30f)) atomicOr(P.err, 1u);
  if (REC) record_u(P, x, y, ux, uy);
  const int nxt = P.parity ^ 1;
#pragma unroll
  for (int j = 0; j < 8; ++j) A[ip_off(P, x + ex_of(j), y + ey_of(j), j, nxt)] = S::enc(d[j], P.scale);
  if (THERMAL) {
    collide_d2q5(g, ux, uy, P);
#pragma unroll
    for (int j = 0; j < 5; ++j) G[ip_off5(P, x + ex5(j), y + ey5(j), j, nxt)] = S::enc(g[j], P.scale);
  }
}

// cells x0 + 1 .. x0 + 4 of a row: one cell, an aligned pair, one cell
template <int PREC>
__device__ __forceinline__ void load_right(const typename Store<PREC>::T* row, int x0, float inv, float o[4]) {
  using S = Store<PREC>;
  o[0] = S::dec(row[x0 + 1], inv);
  S::load2(row + x0 + 2, o + 1, inv);
  o[3] = S::dec(row[x0 + 4], inv);
}

template <int PREC>
__device__ __forceinline__ void store_right(typename Store<PREC>::T* row, int x0, const float v[4], float sc) {
  using S = Store<PREC>;
  row[x0 + 1] = S::enc(v[0], sc);
  S::store2r(row + x0 + 2, make_float2(v[1] * sc, v[2] * sc));
  row[x0 + 4] = S::enc(v[3], sc);
}

// 16-bit storage as words of two cells: the aligned four cells at p (two words), and cells
// p + 1 .. p + 4 (one half-word, one word, one half-word) repacked as (p+1, p+2), (p+3, p+4)
__device__ __forceinline__ void load4w(const void* p, uint32_t w[2]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  w[0] = v.x;
  w[1] = v.y;
}
__device__ __forceinline__ void store4w(void* p, const uint32_t w[2]) { *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]); }
__device__ __forceinline__ void load_right_w(const unsigned short* row, uint32_t w[2]) {
  const uint32_t a = row[1], m = *reinterpret_cast<const uint32_t*>(row + 2), b = row[4];
  w[0] = __byte_perm(a, m, 0x5410);
  w[1] = __byte_perm(m, b, 0x5432);
}
__device__ __forceinline__ void store_right_w(unsigned short* row, const uint32_t w[2]) {
  row[1] = (unsigned short)(w[0] & 0xffffu);
  *reinterpret_cast<uint32_t*>(row + 2) = __byte_perm(w[0], w[1], 0x5432);
  row[4] = (unsigned short)(w[1] >> 16);
}

template <int PAR>
__device__ __forceinline__ constexpr int plane_of(int i) {
  return PAR ? i : (i < 4 ? (i + 2) & 3 : 4 + ((i - 4 + 2) & 3));
}

// Cells of the frame, the groups with a cell on a wall or on the last column (see k_step_ip):
// whole wall rows (y = 0 and ny - 1 when the y sides are not periodic), and in the other rows the
// cells x < L (the first group, when the x sides are not periodic) and x >= R (the groups that
// reach column nx - 1 through their right neighbours).
struct IpFrame {
  int L, R, E, wall_rows;
  int64_t total;
};

__host__ __device__ __forceinline__ IpFrame ip_frame_of(int nx, int ny, int bc_x, int bc_y) {
  IpFrame F;
  F.L = bc_x != BC_PERIODIC ? (nx < 4 ? nx : 4) : 0;
  const int x0e = nx <= 4 ? 0 : (nx - 1) / 4 * 4;  // first group start with x0 + 4 >= nx
  F.R = x0e > F.L ? x0e : F.L;
  F.E = F.L + (nx - F.R);
  F.wall_rows = bc_y != BC_PERIODIC ? 2 : 0;
  F.total = (int64_t)F.wall_rows * nx + (int64_t)(ny - F.wall_rows) * F.E;
  return F;
}

__device__ __forceinline__ void ip_frame_cell(const IpFrame& F, int nx, int ny, int64_t k, int& x, int& y) {
  const int64_t wc = (int64_t)F.wall_rows * nx;
  if (k < wc) {
    y = k < nx ? 0 : ny - 1;
    x = (int)(k < nx ? k : k - nx);
  } else {
    const int64_t r = (k - wc) / F.E;
    const int j = (int)(k - wc - r * F.E);
    y = (int)r + (F.wall_rows ? 1 : 0);
    x = j < F.L ? j : F.R + (j - F.L);
  }
}

// Interior cells of a uniform medium with 16-bit storage, collided two at a time (collide_pair)
// on the stored words, as the A-B step does where it is bound by instruction issue.
template <int PREC, bool HET, bool THERMAL>
constexpr bool kIpPacked = PREC != PREC_FP32 && !HET && !THERMAL;

// Block blk of one in-place step of a lattice: blocks [0, frame_blocks) do the frame cells, one
// per thread, with the generic rules; the others do groups of four cells of one row, gx blocks per
// row, and skip the groups of the frame.
template <int PREC, bool HET, bool THERMAL, int PAR, bool REC>
__device__ __forceinline__ void ip_block(const StepParams& P, int frame_blocks, int gx, int blk) {
  using S = Store<PREC>;
  using T = typename S::T;
  constexpr int C = kIpCells;
  T* __restrict__ A = static_cast<T*>(P.dst);
  T* __restrict__ G = static_cast<T*>(P.gdst);
  if (blk < frame_blocks) {
    const IpFrame F = ip_frame_of(P.nx, P.ny, P.bc_x, P.bc_y);
    const int64_t k = (int64_t)blk * kIpThreads + threadIdx.x;
    if (k >= F.total) return;
    int x, y;
    ip_frame_cell(F, P.nx, P.ny, k, x, y);
    if (!dbg_check(P, x >= 0 && x < P.nx && y >= 0 && y < P.ny)) return;
    ip_cell<PREC, HET, THERMAL, REC>(P, A, G, x, y);
    return;
  }
  const int b = blk - frame_blocks;
  const int y = b / gx;
  const int x0 = ((b - y * gx) * kIpThreads + (int)threadIdx.x) * C;
  if (x0 >= P.nx || !dbg_check(P, y < P.ny)) return;
  const bool edge = (P.bc_x != BC_PERIODIC && x0 == 0) || x0 + C >= P.nx || (P.bc_y != BC_PERIODIC && (y == 0 || y == P.ny - 1));
  if (edge) return;  // a frame group
  // rows y - 1 and y + 1 (periodic wrap; wall rows are frame rows)
  const int ym = y == 0 ? P.ny - 1 : y - 1;
  const int yp = y == P.ny - 1 ? 0 : y + 1;
  const int64_t rm = (int64_t)ym * P.pitch, r0 = (int64_t)y * P.pitch, rp = (int64_t)yp * P.pitch;
  // the slot of population i (see ip_off), as 32-bit element offsets from A (a buffer holds fewer
  // than 2^32 elements; lbm_create checks): plane * pl + y0x (+ the row change dp or dm for the
  // slots of rows y + 1 and y - 1)
  const uint32_t pl = (uint32_t)P.plane;
  const uint32_t y0x = (uint32_t)r0 + (uint32_t)x0;
  const uint32_t dp = (uint32_t)(rp - r0), dm = (uint32_t)(rm - r0);
  if constexpr (kIpPacked<PREC, HET, THERMAL>) {
    unsigned short* const W = reinterpret_cast<unsigned short*>(A);
    uint32_t w[8][2];
    load4w(W + plane_of<PAR>(0) * pl + y0x, w[0]);             // e1 = ( 1, 0): own cells
    load4w(W + plane_of<PAR>(1) * pl + y0x, w[1]);             // e2 = ( 0, 1): own cells
    load_right_w(W + plane_of<PAR>(2) * pl + y0x, w[2]);       // e3 = (-1, 0): cells x + 1 of row y
    load4w(W + (plane_of<PAR>(3) * pl + y0x + dp), w[3]);      // e4 = ( 0,-1): cells of row y + 1
    load4w(W + plane_of<PAR>(4) * pl + y0x, w[4]);             // e5 = ( 1, 1): own cells
    load_right_w(W + (plane_of<PAR>(5) * pl + y0x + dm), w[5]);  // e6 = (-1, 1): cells x + 1 of row y - 1
    load_right_w(W + (plane_of<PAR>(6) * pl + y0x + dp), w[6]);  // e7 = (-1,-1): cells x + 1 of row y + 1
    load4w(W + plane_of<PAR>(7) * pl + y0x, w[7]);             // e8 = ( 1,-1): own cells
    float check = 0.0f;
#pragma unroll
    for (int h = 0; h < C / 2; ++h) {
      float2 dp2[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) dp2[i] = S::w2f(w[i][h]);
      float2 ux, uy;
      collide_pair(dp2, pair_coef_uniform(P.pc), f2(P.pc.u_hx), f2(P.pc.u_hy), P.pc, ux, uy);
      check += (fabsf(ux.x) + fabsf(uy.x)) + (fabsf(ux.y) + fabsf(uy.y));
      if (REC) record_u2(P, x0 + 2 * h, y, ux, uy);
#pragma unroll
      for (int i = 0; i < 8; ++i) w[i][h] = S::f2w(dp2[i]);
    }
    if (!(check < 1e30f)) atomicOr(P.err, 1u);  // non-finite velocity in these cells
    uint32_t b0 = y0x;
    asm volatile("" : "+r"(b0));
    store4w(W + plane_of<PAR>(0) * pl + b0, w[2]);
    store4w(W + plane_of<PAR>(1) * pl + b0, w[3]);
    store_right_w(W + plane_of<PAR>(2) * pl + b0, w[0]);
    store4w(W + (plane_of<PAR>(3) * pl + b0 + dp), w[1]);
    store4w(W + plane_of<PAR>(4) * pl + b0, w[6]);
    store_right_w(W + (plane_of<PAR>(5) * pl + b0 + dm), w[7]);
    store_right_w(W + (plane_of<PAR>(6) * pl + b0 + dp), w[4]);
    store4w(W + plane_of<PAR>(7) * pl + b0, w[5]);
    return;
  } else {
    const float inv = P.inv_scale;
    float4 ph4, k4;
    if (HET) {
      ph4 = __ldg(reinterpret_cast<const float4*>(P.phi + r0 + x0));
      k4 = __ldg(reinterpret_cast<const float4*>(P.K + r0 + x0));
    }
    float d[8][C];
    S::load4(A + plane_of<PAR>(0) * pl + y0x, d[0], inv);             // e1 = ( 1, 0): own cells
    S::load4(A + plane_of<PAR>(1) * pl + y0x, d[1], inv);             // e2 = ( 0, 1): own cells
    load_right<PREC>(A + plane_of<PAR>(2) * pl + y0x, 0, inv, d[2]);  // e3 = (-1, 0): cells x + 1 of row y
    S::load4(A + (plane_of<PAR>(3) * pl + y0x + dp), d[3], inv);      // e4 = ( 0,-1): cells of row y + 1
    S::load4(A + plane_of<PAR>(4) * pl + y0x, d[4], inv);             // e5 = ( 1, 1): own cells
    load_right<PREC>(A + (plane_of<PAR>(5) * pl + y0x + dm), 0, inv, d[5]);  // e6 = (-1, 1): cells x + 1 of row y - 1
    load_right<PREC>(A + (plane_of<PAR>(6) * pl + y0x + dp), 0, inv, d[6]);  // e7 = (-1,-1): cells x + 1 of row y + 1
    S::load4(A + plane_of<PAR>(7) * pl + y0x, d[7], inv);             // e8 = ( 1,-1): own cells
    float g[5][C];
    if (THERMAL) {
      S::load4(G + y0x, g[0], inv);                                    // rest population
      S::load4(G + (PAR ? 1 : 3) * pl + y0x, g[1], inv);               // ( 1, 0): own cells
      S::load4(G + (PAR ? 2 : 4) * pl + y0x, g[2], inv);               // ( 0, 1): own cells
      load_right<PREC>(G + (PAR ? 3 : 1) * pl + y0x, 0, inv, g[3]);    // (-1, 0): cells x + 1
      S::load4(G + ((PAR ? 4 : 2) * pl + y0x + dp), g[4], inv);        // ( 0,-1): row y + 1
    }
    float check = 0.0f, rux = 0.0f, ruy = 0.0f;
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
      if (REC) {  // the record in pairs of cells
        if (c & 1) {
          record_u2(P, x0 + c - 1, y, make_float2(rux, ux), make_float2(ruy, uy));
        } else {
          rux = ux;
          ruy = uy;
        }
      }
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
    if (!(check < 1e30f)) atomicOr(P.err, 1u);  // non-finite velocity in these cells
    // post-collision population opp(i) into the slot population i came from; the offsets are
    // formed again from an opaque copy of y0x rather than kept live through the collision
    uint32_t b0 = y0x;
    asm volatile("" : "+r"(b0));
    const float sc = P.scale;
    S::store4(A + plane_of<PAR>(0) * pl + b0, d[2], sc);
    S::store4(A + plane_of<PAR>(1) * pl + b0, d[3], sc);
    store_right<PREC>(A + plane_of<PAR>(2) * pl + b0, 0, d[0], sc);
    S::store4(A + (plane_of<PAR>(3) * pl + b0 + dp), d[1], sc);
    S::store4(A + plane_of<PAR>(4) * pl + b0, d[6], sc);
    store_right<PREC>(A + (plane_of<PAR>(5) * pl + b0 + dm), 0, d[7], sc);
    store_right<PREC>(A + (plane_of<PAR>(6) * pl + b0 + dp), 0, d[4], sc);
    S::store4(A + plane_of<PAR>(7) * pl + b0, d[5], sc);
    if (THERMAL) {
      S::store4(G + b0, g[0], sc);
      S::store4(G + (PAR ? 1 : 3) * pl + b0, g[3], sc);
      S::store4(G + (PAR ? 2 : 4) * pl + b0, g[4], sc);
      store_right<PREC>(G + (PAR ? 3 : 1) * pl + b0, 0, g[1], sc);
      S::store4(G + ((PAR ? 4 : 2) * pl + b0 + dp), g[2], sc);
    }
  }
}

// Register caps: 8 CTAs of 128 threads per SM for the FP32 flow (64 registers, as the A-B step), 7
// with 16-bit storage (72 registers: 4096^2 FP16 169.1 -> 173.5 GLUPS, 160.9 at 80), 5 with the
// temperature populations (96; at 80 the FP32 thermal step spills).
template <int PREC, bool HET, bool THERMAL, int PAR, bool REC>
__global__ void __launch_bounds__(kIpThreads, THERMAL ? 5 : (PREC == PREC_FP32 ? 8 : 7)) k_step_ip(const StepParams P, int frame_blocks, int gx) {
  ip_block<PREC, HET, THERMAL, PAR, REC>(P, frame_blocks, gx, (int)blockIdx.x);
}

// Batched ensembles with in-place streaming: one CTA per work item, the item's lattice from a
// per-item table and the lattice's parameters staged once per CTA in shared memory, as in the A-B
// batched step; the lattices' items are those of k_step_ip, concatenated (item_start ascending).
template <int PREC, int PAR>
__global__ void __launch_bounds__(kIpThreads, 8) k_step_ip_batch(const StepParams* __restrict__ Pd, const int64_t* __restrict__ item_start,
                                                               const int* __restrict__ item_lattice) {
  __shared__ StepParams sP;
  const int d = item_lattice[blockIdx.x];
  {
    static_assert(sizeof(StepParams) % 8 == 0, "parameters are copied as 8-byte words");
    const unsigned long long* from = reinterpret_cast<const unsigned long long*>(Pd + d);
    unsigned long long* to = reinterpret_cast<unsigned long long*>(&sP);
    for (int i = threadIdx.x; i < (int)(sizeof(StepParams) / 8); i += kIpThreads) to[i] = from[i];
  }
  __syncthreads();
  const IpFrame F = ip_frame_of(sP.nx, sP.ny, sP.bc_x, sP.bc_y);
  const int frame_blocks = (int)((F.total + kIpThreads - 1) / kIpThreads);
  const int gx = ((sP.nx + kIpCells - 1) / kIpCells + kIpThreads - 1) / kIpThreads;
  ip_block<PREC, true, false, PAR, false>(sP, frame_blocks, gx, (int)((int64_t)blockIdx.x - item_start[d]));
}

template <int PREC, bool HET, bool THERMAL>
static cudaError_t launch_ip_t(const StepParams& P, cudaStream_t s) {
  const IpFrame F = ip_frame_of(P.nx, P.ny, P.bc_x, P.bc_y);
  const int frame_blocks = (int)((F.total + kIpThreads - 1) / kIpThreads);
  const int groups = (P.nx + kIpCells - 1) / kIpCells;
  const int gx = (groups + kIpThreads - 1) / kIpThreads;
  const long long blocks = (long long)frame_blocks + (long long)gx * P.ny;
  if (P.edge) {  // the boundary nodes' states, before the step overwrites their neighbours' slots
    const int64_t threads = 8 * 2 * ((int64_t)P.nx + P.ny);
    k_edge_ip<PREC, HET, THERMAL><<<(unsigned)((threads + 127) / 128), 128, 0, s>>>(P);
  }
  // the variant that records u runs once per lbm_step call
  if (P.urec) {
    if (P.parity)
      k_step_ip<PREC, HET, THERMAL, 1, true><<<(unsigned)blocks, kIpThreads, 0, s>>>(P, frame_blocks, gx);
    else
      k_step_ip<PREC, HET, THERMAL, 0, true><<<(unsigned)blocks, kIpThreads, 0, s>>>(P, frame_blocks, gx);
  } else if (P.parity) {
    k_step_ip<PREC, HET, THERMAL, 1, false><<<(unsigned)blocks, kIpThreads, 0, s>>>(P, frame_blocks, gx);
  } else {
    k_step_ip<PREC, HET, THERMAL, 0, false><<<(unsigned)blocks, kIpThreads, 0, s>>>(P, frame_blocks, gx);
  }
  return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_ip_p(const StepParams& P, bool het, bool thermal, cudaStream_t s) {
  if (thermal) return het ? launch_ip_t<PREC, true, true>(P, s) : launch_ip_t<PREC, false, true>(P, s);
  return het ? launch_ip_t<PREC, true, false>(P, s) : launch_ip_t<PREC, false, false>(P, s);
}

// work items (CTAs) of one in-place step of a lattice
int64_t inplace_items(int nx, int ny, int bc_x, int bc_y) {
  const IpFrame F = ip_frame_of(nx, ny, bc_x, bc_y);
  const int64_t gx = ((nx + kIpCells - 1) / kIpCells + kIpThreads - 1) / kIpThreads;
  return (F.total + kIpThreads - 1) / kIpThreads + gx * ny;
}

cudaError_t launch_step_batch_inplace(const StepParams* Pd, const int64_t* item_start, const int* item_lattice, int64_t total, int prec,
                                      int parity, cudaStream_t s) {
#define LBM_IPB(PR)                                                                                   \
  do {                                                                                                \
    if (parity) k_step_ip_batch<PR, 1><<<(unsigned)total, kIpThreads, 0, s>>>(Pd, item_start, item_lattice); \
    else k_step_ip_batch<PR, 0><<<(unsigned)total, kIpThreads, 0, s>>>(Pd, item_start, item_lattice);        \
  } while (0)
  if (prec == PREC_FP32) LBM_IPB(PREC_FP32);
  else if (prec == PREC_FP16) LBM_IPB(PREC_FP16);
  else LBM_IPB(PREC_BF16);
#undef LBM_IPB
  return cudaGetLastError();
}

cudaError_t launch_step_inplace(const StepParams& P, int prec, bool het, bool thermal, cudaStream_t s) {
  switch (prec) {
    case PREC_FP32: return launch_ip_p<PREC_FP32>(P, het, thermal, s);
    case PREC_FP16: return launch_ip_p<PREC_FP16>(P, het, thermal, s);
    default: return launch_ip_p<PREC_BF16>(P, het, thermal, s);
  }
}

// --------------------------------------------------------------------------------------------
// Writing a pre-collision state f(x, t) into the in-place layout of the current parity: every
// population goes to the slot that the next step's pull reads it from (for a link that crosses a
// wall, the parked slot, holding the value minus the moving-wall term, or for an isothermal wall
// the anti-bounce-back inverse).
// --------------------------------------------------------------------------------------------
// flow: f (dense [8][ny][nx] float32, full populations) or, if f is null, the equilibrium of
// Eq. 22 at (p0, u0) (phi p = p0 when phip_uniform, else phi p0)
template <int PREC, bool HET>
__global__ void k_put_flow_ip(const StepParams P, const float* __restrict__ f, float p0, float ux0, float uy0, int phip_uniform) {
  using S = Store<PREC>;
  using T = typename S::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  T* A = static_cast<T*>(P.dst);
  float d[8];
  if (f) {
    const int64_t dense = (int64_t)P.nx * P.ny, o = (int64_t)y * P.nx + x;
    for (int i = 0; i < 8; ++i) d[i] = f[i * dense + o] - 3.0f * w_of(i) * P.p_rest;
  } else {
    const Coef c = coef_at<HET>(P, x, y);
    feq_dev_d2q8((phip_uniform ? p0 : c.phi * p0) - P.p_rest, ux0, uy0, c.inv_phi, P.rho0, d);
  }
  for (int i = 0; i < 8; ++i) {
    int w;
    const int64_t at = ip_source(P, x, y, i, w);
    A[at] = S::enc(w < 0 ? d[i] : d[i] - wall_term(P, i, w), P.scale);
  }
}

// temperature: g (dense [5][ny][nx]) or, if g is null, the equilibrium of Eq. B.6 at T_init, u = 0
template <int PREC>
__global__ void k_put_thermal_ip(const StepParams P, const float* __restrict__ g, float T_init) {
  using S = Store<PREC>;
  using T = typename S::T;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  T* G = static_cast<T*>(P.gdst);
  float z[5];
  if (g) {
    const int64_t dense = (int64_t)P.nx * P.ny, o = (int64_t)y * P.nx + x;
    for (int i = 0; i < 5; ++i) z[i] = g[i * dense + o] - 0.2f * P.T0;
  } else {
    geq_dev(P, T_init, 0.0f, 0.0f, z);
  }
  for (int i = 0; i < 5; ++i) {
    int w;
    const int64_t at = ip_source5(P, x, y, i, w);
    // inverse of the pull: z = v (bounce-back) or z = -v + 2 (T_w - T0) / 5 (anti-bounce-back)
    const float v = (w < 0 || !P.Tdir[w]) ? z[i] : (0.4f * (P.Tw[w] - P.T0) - z[i]);
    G[at] = S::enc(v, P.scale);
  }
}

cudaError_t launch_put_inplace(const StepParams& P, int prec, bool het, const float* f, const float* g, bool flow, bool temp,
                               float p0, float ux0, float uy0, int phip_uniform, float T_init, cudaStream_t s) {
  const dim3 grid((P.nx + 127) / 128, P.ny);
  if (flow) {
#define LBM_PUT(PR)                                                                                       \
  do {                                                                                                    \
    if (het) k_put_flow_ip<PR, true><<<grid, 128, 0, s>>>(P, f, p0, ux0, uy0, phip_uniform);            \
    else k_put_flow_ip<PR, false><<<grid, 128, 0, s>>>(P, f, p0, ux0, uy0, phip_uniform);               \
  } while (0)
    if (prec == PREC_FP32) LBM_PUT(PREC_FP32);
    else if (prec == PREC_FP16) LBM_PUT(PREC_FP16);
    else LBM_PUT(PREC_BF16);
#undef LBM_PUT
  }
  if (temp) {
    if (prec == PREC_FP32) k_put_thermal_ip<PREC_FP32><<<grid, 128, 0, s>>>(P, g, T_init);
    else if (prec == PREC_FP16) k_put_thermal_ip<PREC_FP16><<<grid, 128, 0, s>>>(P, g, T_init);
    else k_put_thermal_ip<PREC_BF16><<<grid, 128, 0, s>>>(P, g, T_init);
  }
  return cudaGetLastError();
}

}  // namespace lbm
