// Tiling shared by the forward and adjoint stream-collide kernels: a thread owns a group of
// kCellsPerThread consecutive cells of one row; rows are read as aligned vectors and the one-cell
// x-shift of a population comes from the neighbouring lane (warp shuffle); the groups touching a
// wall row or the first/last column form the "frame" and are handled by dedicated work items.
#pragma once

#include "lbm_device.cuh"

namespace lbm {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kStepThreads = 128;
constexpr int kCellsPerThread = 4;

// out[c] = row[x0 + c - SH] for c = 0..3 (SH = +1: pull from x-1, SH = -1: from x+1, 0: aligned);
// RAW: the stored values as they are (no storage scale applied).
template <int PREC, int SH, bool RAW = false>
__device__ __forceinline__ void gather4(const typename Store<PREC>::T* __restrict__ row, int xl, int pitch, int lane,
                                        float inv, float out[4]) {
  using S = Store<PREC>;
  float v[4];
  if (RAW) S::load4r(row + xl, v);
  else S::load4(row + xl, v, inv);
  if (SH == 0) {
    out[0] = v[0]; out[1] = v[1]; out[2] = v[2]; out[3] = v[3];
  } else if (SH == 1) {
    float left = __shfl_up_sync(kFull, v[3], 1);
    if (lane == 0) {
      const typename S::T e = row[xl > 0 ? xl - 1 : 0];
      left = RAW ? S::decr(e) : S::dec(e, inv);
    }
    out[0] = left; out[1] = v[0]; out[2] = v[1]; out[3] = v[2];
  } else {
    float right = __shfl_down_sync(kFull, v[0], 1);
    if (lane == 31) {
      const typename S::T e = row[xl + 4 < pitch ? xl + 4 : pitch - 1];
      right = RAW ? S::decr(e) : S::dec(e, inv);
    }
    out[0] = v[1]; out[1] = v[2]; out[2] = v[3]; out[3] = right;
  }
}

// 16-bit storage kept as stored: the four values of gather4 as two 32-bit words (cells 0-1 and
// 2-3, first cell in the low half); the one-cell shifts are byte permutes of neighbouring words.
template <int PREC, int SH>
__device__ __forceinline__ void gather4w(const typename Store<PREC>::T* __restrict__ row, int xl, int pitch, int lane,
                                         uint32_t out[2]) {
  using S = Store<PREC>;
  static_assert(sizeof(typename S::T) == 2, "16-bit storage");
  const uint2 v = *reinterpret_cast<const uint2*>(row + xl);
  if (SH == 0) {
    out[0] = v.x; out[1] = v.y;
  } else if (SH == 1) {  // cells x - 1: (left, c0), (c1, c2)
    uint32_t lw = __shfl_up_sync(kFull, v.y, 1);  // its high half is the left neighbour's last cell
    if (lane == 0) lw = S::bits(row[xl > 0 ? xl - 1 : 0]) << 16;
    out[0] = __byte_perm(lw, v.x, 0x5432);
    out[1] = __byte_perm(v.x, v.y, 0x5432);
  } else {  // cells x + 1: (c1, c2), (c3, right)
    uint32_t rw = __shfl_down_sync(kFull, v.x, 1);  // its low half is the right neighbour's first cell
    if (lane == 31) rw = S::bits(row[xl + 4 < pitch ? xl + 4 : pitch - 1]);
    out[0] = __byte_perm(v.x, v.y, 0x5432);
    out[1] = __byte_perm(v.y, rw, 0x5432);
  }
}

// The same for a pair of cells: out[c] = row[x0 + c - SH], c = 0, 1 (x0 even, 2-element aligned).
template <int PREC, int SH>
__device__ __forceinline__ void gather2(const typename Store<PREC>::T* __restrict__ row, int xl, int pitch, int lane, float inv,
                                        float out[2]) {
  using S = Store<PREC>;
  float v[2];
  S::load2(row + xl, v, inv);
  if (SH == 0) {
    out[0] = v[0]; out[1] = v[1];
  } else if (SH == 1) {
    float left = __shfl_up_sync(kFull, v[1], 1);
    if (lane == 0) left = S::dec(row[xl > 0 ? xl - 1 : 0], inv);
    out[0] = left; out[1] = v[0];
  } else {
    float right = __shfl_down_sync(kFull, v[0], 1);
    if (lane == 31) right = S::dec(row[xl + 2 < pitch ? xl + 2 : pitch - 1], inv);
    out[0] = v[1]; out[1] = right;
  }
}

// Frame of the lattice: the groups of C cells that contain a wall-row cell or a cell of the first
// or last column (the last group of a row also holds the row padding).  Their cells are gathered
// with every boundary rule (pull_one: halfway bounce-back with wall velocity, periodic wrap,
// pressure columns), collided and stored by dedicated blocks; the main blocks skip them.
struct Frame {
  int groups_per_row;  // G = ceil(nx / C)
  int cols;            // frame groups per non-wall row: 1 if G == 1, else 2
  int wall_rows;       // 1 if the bottom and top rows are walls
  int count;           // number of frame groups
};

__host__ __device__ inline Frame frame_of(int nx, int ny, int bc_y, int C) {
  Frame f;
  f.groups_per_row = (nx + C - 1) / C;
  f.cols = f.groups_per_row == 1 ? 1 : 2;
  f.wall_rows = (bc_y == BC_WALL || bc_y == BC_NEE) ? 1 : 0;
  f.count = (f.wall_rows ? 2 * f.groups_per_row : 0) + f.cols * (ny - (f.wall_rows ? 2 : 0));
  return f;
}

// Work items of one lattice for CTAs of nt threads: the frame items first, then the main items.
// Row-aligned tiling: a row of G = ceil(nx / C) groups takes gx = ceil(G / nt) items when G > nt;
// shorter rows are packed rows_per_item = nt / G to an item (thread t of the item: row t / G,
// group t % G).  Flat tiling: the ny G groups in row-major order, nt consecutive groups per item,
// so that an item may span the end of one row and the start of the next; only the lattice's last
// item is ragged.  (Within a warp the one-cell shifts then also cross a row end, between the last
// group of a row and the first of the next: both are frame groups, whose main-path results are
// not stored.)
struct Tiling {
  int frame_blocks, gx, rows_per_item, groups, flat;
};

// Row and column of frame cell k (frame group k / C, cell k % C of the group).
__device__ __forceinline__ bool frame_cell(const Frame& F, int ny, int k, int& x, int& y) {
  const int grp = k / kCellsPerThread;
  if (grp >= F.count) return false;
  int x0;
  if (F.wall_rows && grp < 2 * F.groups_per_row) {
    y = grp < F.groups_per_row ? 0 : ny - 1;
    x0 = (grp % F.groups_per_row) * kCellsPerThread;
  } else {
    const int k2 = grp - (F.wall_rows ? 2 * F.groups_per_row : 0);
    y = k2 / F.cols + F.wall_rows;
    x0 = (k2 % F.cols == 0) ? 0 : (F.groups_per_row - 1) * kCellsPerThread;
  }
  x = x0 + (k - grp * kCellsPerThread);
  return true;
}

__host__ __device__ inline Tiling tiling_of(int nx, int ny, int bc_y, int nt, bool flat = false) {
  Tiling t;
  t.flat = flat ? 1 : 0;
  t.groups = (nx + kCellsPerThread - 1) / kCellsPerThread;
  const Frame F = frame_of(nx, ny, bc_y, kCellsPerThread);
  t.frame_blocks = (int)(((int64_t)F.count * kCellsPerThread + nt - 1) / nt);  // one thread per frame cell
  if (t.groups <= nt) {
    t.gx = 1;
    t.rows_per_item = nt / t.groups;
  } else {
    t.gx = (t.groups + nt - 1) / nt;
    t.rows_per_item = 1;
  }
  return t;
}

__host__ __device__ inline int64_t main_items(const Tiling& t, int ny, int nt) {
  if (t.flat) return ((int64_t)ny * t.groups + nt - 1) / nt;
  return t.rows_per_item > 1 ? (int64_t)((ny + t.rows_per_item - 1) / t.rows_per_item) : (int64_t)t.gx * ny;
}

// Row and first cell of thread `tid` in main item b; false for a thread with no group (it still
// takes part in the loads and shuffles, on a clamped row, and stores nothing).
__device__ __forceinline__ bool main_group(const Tiling& t, int ny, int nt, int b, int tid, int& x0, int& y) {
  if (t.flat) {
    const int64_t g = (int64_t)b * nt + tid;
    y = (int)(g / t.groups);
    x0 = (int)(g - (int64_t)y * t.groups) * kCellsPerThread;
    const bool ok = y < ny;
    if (!ok) y = ny - 1;
    return ok;
  }
  if (t.rows_per_item > 1) {
    const int r = tid / t.groups;
    y = b * t.rows_per_item + r;
    x0 = (tid - r * t.groups) * kCellsPerThread;
    const bool ok = r < t.rows_per_item && y < ny;
    if (!ok) y = ny - 1;
    return ok;
  }
  y = b / t.gx;
  x0 = ((b - y * t.gx) * nt + tid) * kCellsPerThread;
  return true;
}

}  // namespace lbm
