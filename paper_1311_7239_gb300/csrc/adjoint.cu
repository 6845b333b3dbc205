// Discrete adjoint of the fused D2Q8 porous MRT-LB step (Liu & He, arXiv 1311.7239, Eqs. 3-20):
// gradients of a scalar loss of the state after T steps with respect to the per-cell
// log-permeability l = log K and porosity phi (theta of Eq. 3 and Eq. 4).
//
// Forward map in pre-collision variables: z(t+1) = N(P(C(z(t); theta)); theta), z(0) = N(f_eq(theta)),
// with C the collision (Eq. 14 as d+ = d + M^-1 k, k = m+ - m), P the pull streaming with its wall
// rules (Eq. 15) and N the boundary nodes: the pressure columns, then the wall nodes of the sides
// with non-equilibrium extrapolation (Sec. 3's wall treatment), both f_b = f_eq(p_b, u_b; phi_b) +
// f_nb - f_eq(p_nb, u_nb; phi_nb) from the inner neighbour nb.  The adjoint state
// nu(t) = dL/dz(t) obeys nu(t) = J_C(z(t))^T P^T J_N^T nu(t+1); every piece is differentiated
// here by hand in reverse mode:
//   - P^T is the reversed link table (a gather of nu from x + e_i, or from the opposite slot
//     through a wall); the moving-wall term is a constant and has no derivative.
//   - J_C^T mu = mu + M^T kbar, kbar = (dk/dm)^T w, w = M^-T mu, through Eq. 11-14 (m_eq, S),
//     Eq. 3 (F), Eq. 20 (phi p) and the root of Eqs. 18-19 (u, |u|).  At |v| = 0 the derivative
//     of |v| is taken as 0 (the one-sided limit of the smooth part of Eq. 18).
//   - J_N^T moves the adjoint of each wall node (k_adj_wall), then of each pressure-column cell
//     (k_adj_nee), onto its inner neighbour.
// theta enters through phi (Eq. 3, 11, 16, 19, 20 and F_phi of Eq. 4) and K (Eq. 3, 19); with
// c_lin = phi nu / K and c_nl = phi F_phi / sqrt(K) = 1.75 / sqrt(150 phi K):
//   dc_lin/dl = -c_lin, dc_lin/dphi = c_lin / phi, dc_nl/dl = -c_nl / 2, dc_nl/dphi = -c_nl / (2 phi).
// Per-step gradient terms are summed in FP32 over at most kAdjFold steps and then folded into FP64
// totals (k_adj_fold); the adjoint state is stored in FP32 planes [8][ny][pitch].
#include "lbm_device.cuh"
#include "lbm_internal.h"
#include "tiles.cuh"

namespace lbm {

// Reverse of velocity_from_j: adjoints (ubx, uby) of u and umb of |u| -> adjoints of jx, jy and
// of the coefficients c_lin, c_nl and phi (through phi a / 2).
struct VelBar {
  float jx, jy, clin, cnl, phi;
};

// Forward quantities of Eqs. 18-19 kept for the reverse pass (velocity_from_j's intermediates).
struct VelFwd {
  float vx, vy, vmag, sR, inv, l0, l1;
};

__device__ __forceinline__ VelFwd velocity_fwd(float jx, float jy, const Coef& c, float ax, float ay, float inv_rho0) {
  VelFwd f;
  f.vx = jx * inv_rho0 + 0.5f * c.phi * ax;
  f.vy = jy * inv_rho0 + 0.5f * c.phi * ay;
  f.l0 = 0.5f + 0.25f * c.c_lin;
  f.l1 = 0.5f * c.c_nl;
  f.vmag = fast_sqrt(f.vx * f.vx + f.vy * f.vy);
  f.sR = fast_sqrt(f.l0 * f.l0 + f.l1 * f.vmag);
  f.inv = fast_rcp(f.l0 + f.sR);
  return f;
}

__device__ __forceinline__ VelBar velocity_vjp(const VelFwd& f, float inv_rho0, float ax, float ay, float ubx, float uby, float umb) {
  const float vx = f.vx, vy = f.vy, vmag = f.vmag, sR = f.sR, inv = f.inv, l0 = f.l0, l1 = f.l1;
  float vbx = ubx * inv, vby = uby * inv;
  float inv_bar = ubx * vx + uby * vy + umb * vmag;
  float vmag_bar = umb * inv;
  const float D_bar = -inv * inv * inv_bar;
  const float R_bar = D_bar * 0.5f * fast_rcp(sR);
  const float l0_bar = D_bar + 2.0f * l0 * R_bar;
  const float l1_bar = vmag * R_bar;
  vmag_bar += l1 * R_bar;
  if (vmag > 0.0f) {
    const float iv = fast_rcp(vmag);
    vbx += vmag_bar * vx * iv;
    vby += vmag_bar * vy * iv;
  }
  VelBar o;
  o.jx = vbx * inv_rho0;
  o.jy = vby * inv_rho0;
  o.phi = 0.5f * (ax * vbx + ay * vby);
  o.clin = 0.25f * l0_bar;
  o.cnl = 0.5f * l1_bar;
  return o;
}

__device__ __forceinline__ VelBar velocity_vjp(float jx, float jy, const Coef& c, float ax, float ay, float inv_rho0, float ubx,
                                               float uby, float umb) {
  return velocity_vjp(velocity_fwd(jx, jy, c, ax, ay, inv_rho0), inv_rho0, ax, ay, ubx, uby, umb);
}

// theta-gradients from the adjoints of c_lin, c_nl, 1/phi and phi itself.
__device__ __forceinline__ void theta_bar(const Coef& c, float clin_bar, float cnl_bar, float iphi_bar, float phi_bar, float& g_l,
                                          float& g_phi) {
  g_l += -c.c_lin * clin_bar - 0.5f * c.c_nl * cnl_bar;
  g_phi += phi_bar - c.inv_phi * c.inv_phi * iphi_bar + c.c_lin * c.inv_phi * clin_bar - 0.5f * c.c_nl * c.inv_phi * cnl_bar;
}

// nu = J_C(z)^T mu and the theta-gradient (dC/dtheta)^T mu of one cell.
__device__ void collide_vjp(const float z[8], const Coef& c, float ax, float ay, const StepParams& P, const float mu[8], float nu[8],
                            float& g_l, float& g_phi) {
  const float rho0 = P.rho0;
  // forward quantities (as collide_d2q8)
  const float a13 = z[0] + z[2], a24 = z[1] + z[3];
  const float d13 = z[0] - z[2], d24 = z[1] - z[3];
  const float s57 = z[4] + z[6], s68 = z[5] + z[7];
  const float t57 = z[4] - z[6], t68 = z[5] - z[7];
  const float m1 = a13 + a24 + s57 + s68;
  const float m3 = d13 + (t57 - t68), m5 = d24 + (t57 + t68);
  // u = v / (l0 + sqrt(l0^2 + l1 |v|)) (Eqs. 18-19), its intermediates kept for the reverse pass
  const VelFwd vf = velocity_fwd(m3, m5, c, ax, ay, P.inv_rho0);
  const float ux = vf.vx * vf.inv, uy = vf.vy * vf.inv, umag = vf.vmag * vf.inv;
  const float usq = ux * ux + uy * uy;
  const float drag = c.c_lin + c.c_nl * umag;
  const float Fx = -drag * ux + c.phi * ax;
  const float Fy = -drag * uy + c.phi * ay;
  const float ip = c.inv_phi;
  (void)m1;
  // w = M^-T mu = diag(1/8, 1/8, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4) M mu (w1 is not needed: k1 = 0)
  const float b13 = mu[0] - mu[2], b24 = mu[1] - mu[3];
  const float bx = mu[4] - mu[5] - mu[6] + mu[7], by = mu[4] + mu[5] - mu[6] - mu[7];
  const float w2 = (-(mu[0] + mu[1] + mu[2] + mu[3]) + (mu[4] + mu[5] + mu[6] + mu[7])) * 0.125f;
  const float w3 = (b13 + bx) * (1.0f / 6.0f), w4 = (-2.0f * b13 + bx) * (1.0f / 12.0f);
  const float w5 = (b24 + by) * (1.0f / 6.0f), w6 = (-2.0f * b24 + by) * (1.0f / 12.0f);
  const float w7 = (mu[0] - mu[1] + mu[2] - mu[3]) * 0.25f, w8 = (mu[4] - mu[5] + mu[6] - mu[7]) * 0.25f;
  const float s_e = P.s_e, s_q = P.s_q, s_v = c.s_v, hv = 1.0f - 0.5f * s_v;
  float mb1 = 0.f, mb2 = 0.f, mb3 = 0.f, mb4 = 0.f, mb5 = 0.f, mb6 = 0.f, mb7 = 0.f, mb8 = 0.f;
  float ubx = 0.f, uby = 0.f, Fbx = 0.f, Fby = 0.f, Pb = 0.f, S2b = 0.f, ipb = 0.f, phib = 0.f;
  // k2 = -s_e (m2 + phi p) + (1 - s_e/2) S2
  mb2 += -s_e * w2;
  Pb += -s_e * w2;
  S2b += (1.0f - 0.5f * s_e) * w2;
  // k3 = rho0 F_x ; k4 = -s_q (m4 + m3) - rho0 F_x
  Fbx += rho0 * w3 - rho0 * w4;
  mb4 += -s_q * w4;
  mb3 += -s_q * w4;
  // k5 = rho0 F_y ; k6 = -s_q (m6 + m5) - rho0 F_y
  Fby += rho0 * w5 - rho0 * w6;
  mb6 += -s_q * w6;
  mb5 += -s_q * w6;
  // k7 = -s_v m7 + s_v rho0 (ux^2 - uy^2)/phi + hv 2 rho0 (ux Fx - uy Fy)/phi
  mb7 += -s_v * w7;
  ubx += w7 * 2.0f * rho0 * ip * (s_v * ux + hv * Fx);
  uby += -w7 * 2.0f * rho0 * ip * (s_v * uy + hv * Fy);
  Fbx += w7 * 2.0f * hv * rho0 * ux * ip;
  Fby += -w7 * 2.0f * hv * rho0 * uy * ip;
  ipb += w7 * rho0 * (s_v * (ux * ux - uy * uy) + 2.0f * hv * (ux * Fx - uy * Fy));
  // k8 = -s_v m8 + s_v rho0 ux uy/phi + hv rho0 (ux Fy + uy Fx)/phi
  mb8 += -s_v * w8;
  ubx += w8 * rho0 * ip * (s_v * uy + hv * Fy);
  uby += w8 * rho0 * ip * (s_v * ux + hv * Fx);
  Fby += w8 * hv * rho0 * ux * ip;
  Fbx += w8 * hv * rho0 * uy * ip;
  ipb += w8 * rho0 * (s_v * ux * uy + hv * (ux * Fy + uy * Fx));
  // S2 = 0.8 rho0 (u . F) / phi
  ubx += S2b * 0.8f * rho0 * Fx * ip;
  uby += S2b * 0.8f * rho0 * Fy * ip;
  Fbx += S2b * 0.8f * rho0 * ux * ip;
  Fby += S2b * 0.8f * rho0 * uy * ip;
  ipb += S2b * 0.8f * rho0 * (ux * Fx + uy * Fy);
  // phi p (deviation) = 0.6 m1 - 0.4 rho0 |u|^2 / phi
  mb1 += 0.6f * Pb;
  ubx += -0.8f * rho0 * ux * ip * Pb;
  uby += -0.8f * rho0 * uy * ip * Pb;
  ipb += -0.4f * rho0 * usq * Pb;
  // F = -(c_lin + c_nl |u|) u + phi a
  ubx += -drag * Fbx;
  uby += -drag * Fby;
  const float drag_b = -(ux * Fbx + uy * Fby);
  float clin_b = drag_b;
  float cnl_b = umag * drag_b;
  const float umag_b = c.c_nl * drag_b;
  phib += ax * Fbx + ay * Fby;
  // u, |u| from j (Eqs. 18-19)
  const VelBar vb = velocity_vjp(vf, P.inv_rho0, ax, ay, ubx, uby, umag_b);
  mb3 += vb.jx;
  mb5 += vb.jy;
  clin_b += vb.clin;
  cnl_b += vb.cnl;
  phib += vb.phi;
  // nu = mu + M^T mbar
  const float A = mb1 - mb2, B = mb1 + mb2;
  const float X = mb3 - 2.0f * mb4, Y = mb5 - 2.0f * mb6;
  const float Px = mb3 + mb4, Py = mb5 + mb6;
  nu[0] = mu[0] + A + X + mb7;
  nu[1] = mu[1] + A + Y - mb7;
  nu[2] = mu[2] + A - X + mb7;
  nu[3] = mu[3] + A - Y - mb7;
  nu[4] = mu[4] + B + Px + Py + mb8;
  nu[5] = mu[5] + B - Px + Py - mb8;
  nu[6] = mu[6] + B - Px - Py + mb8;
  nu[7] = mu[7] + B + Px - Py - mb8;
  theta_bar(c, clin_b, cnl_b, ipb, phib, g_l, g_phi);
}

// pre-collision state of a cell gathered from a post-collision buffer (wall nodes and pressure
// columns included)
template <int PREC, bool HET>
__device__ __forceinline__ void gather_z(const StepParams& P, const void* buf, int x, int y, float z[8]) {
  gather_cell<PREC, HET>(P, static_cast<const typename Store<PREC>::T*>(buf), x, y, z);
}

// --------------------------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------------------------
struct AdjArgs {
  const float* nu_in;  // nu(t+1) after J_N^T (planes [8][ny][pitch])
  float* nu_out;       // nu(t)
  float* g_l;          // dL/dlog K  [ny][pitch], FP32 partial sums (folded into FP64 by k_adj_fold)
  float* g_phi;        // dL/dphi    [ny][pitch], likewise
};

// Seed: nu(T) = dL/dz(T) and the explicit theta-gradient of the loss; per-block loss partials.
// kind 0: L = sum_y u_x(nx-1, y); kind 1: L = 1/2 sum |u - u*|^2.
template <int PREC, bool HET>
__global__ void k_adj_seed(const StepParams P, AdjArgs A, int kind, const float* __restrict__ tux, const float* __restrict__ tuy,
                           double* __restrict__ partial) {
  double lsum = 0.0;
  const int64_t n = (int64_t)P.nx * P.ny;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(k / P.nx), x = (int)(k - (int64_t)y * P.nx);
    float z[8];
    gather_z<PREC, HET>(P, P.src, x, y, z);
    const Coef c = coef_at<HET>(P, x, y);
    const float jx = (z[0] - z[2]) + (z[4] - z[5] - z[6] + z[7]);
    const float jy = (z[1] - z[3]) + (z[4] + z[5] - z[6] - z[7]);
    float ux, uy, umag;
    velocity_from_j(jx, jy, c, P.ax, P.ay, P.inv_rho0, ux, uy, umag);
    float ubx = 0.f, uby = 0.f;
    if (kind == 0) {
      if (x == P.nx - 1) {
        lsum += ux;
        ubx = 1.0f;
      }
    } else {
      const float ex = ux - tux[k], ey = uy - tuy[k];
      lsum += 0.5 * ((double)ex * ex + (double)ey * ey);
      ubx = ex;
      uby = ey;
    }
    float nu[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float gl = 0.0f, gp = 0.0f;
    if (ubx != 0.0f || uby != 0.0f) {
      const VelBar vb = velocity_vjp(jx, jy, c, P.ax, P.ay, P.inv_rho0, ubx, uby, 0.0f);
#pragma unroll
      for (int i = 0; i < 8; ++i) nu[i] = (float)ex_of(i) * vb.jx + (float)ey_of(i) * vb.jy;
      theta_bar(c, vb.clin, vb.cnl, 0.0f, vb.phi, gl, gp);
    }
    const int64_t o = (int64_t)y * P.pitch + x;
#pragma unroll
    for (int i = 0; i < 8; ++i) A.nu_out[i * P.plane + o] = nu[i];
    A.g_l[o] += gl;
    A.g_phi[o] += gp;
  }
  // block sum of the loss
  __shared__ double sh[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_adj_loss_total(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nblocks; ++i) s += partial[i];
    out[0] = s;
  }
}

// J_N^T in place on nu: eight lanes per row and pressure column, lane i holding population i
// (sums over i are reductions within the lane group); when nx < 4 both columns share their
// neighbour column, and one group per row does both in turn.  z(nb) is gathered from `buf`, the
// post-collision buffer whose gather is the state at which N was applied.
__device__ __forceinline__ float group8_sum(float v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 1);
  v += __shfl_xor_sync(mask, v, 2);
  v += __shfl_xor_sync(mask, v, 4);
  return v;
}

template <int PREC, bool HET>
__global__ void k_adj_nee(const StepParams P, const void* buf, float* __restrict__ nu, float* __restrict__ g_l,
                          float* __restrict__ g_phi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int grp = t >> 3, i = t & 7;
  const bool shared_nb = P.nx < 4;
  const int y = shared_nb ? grp : grp >> 1;
  if (y >= P.ny) return;  // whole lane groups leave together
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  using T = typename Store<PREC>::T;
  const float ex = (float)ex_of(i), ey = (float)ey_of(i), w = w_of(i);
  const int s0 = shared_nb ? 0 : (grp & 1), s1 = shared_nb ? 2 : s0 + 1;
  for (int side = s0; side < s1; ++side) {
    const int xb = side ? P.nx - 1 : 0, xn = side ? P.nx - 2 : 1;
    const float pb = side ? P.p_out : P.p_in;
    const int64_t ob = (int64_t)y * P.pitch + xb, on = (int64_t)y * P.pitch + xn;
    const float nbi = nu[i * P.plane + ob];
    nu[i * P.plane + ob] = 0.0f;
    const float zi = pull_one<PREC>(P, static_cast<const T*>(buf), xn, y, i);
    const Coef cn = coef_at<HET>(P, xn, y);
    const Coef cb = coef_at<HET>(P, xb, y);
    const float jx = group8_sum(ex * zi, gm), jy = group8_sum(ey * zi, gm);
    float ux, uy, umag;
    velocity_from_j(jx, jy, cn, P.ax, P.ay, P.inv_rho0, ux, uy, umag);
    const float usq = ux * ux + uy * uy;
    const float rho0 = P.rho0;
    // N_b,i = z_nb,i + 3 w_i (phi_b p_b - phi_n p_n) + rho0 w_i (4.5 (e_i.u)^2 - 1.5 |u|^2)(1/phi_b - 1/phi_n)
    const float wi = w * nbi;
    const float eu = ex * ux + ey * uy;
    const float W = group8_sum(wi, gm);
    const float WA = group8_sum(wi * (4.5f * eu * eu - 1.5f * usq), gm);
    const float gux = group8_sum(wi * (9.0f * eu * ex - 3.0f * ux), gm);
    const float guy = group8_sum(wi * (9.0f * eu * ey - 3.0f * uy), gm);
    const float diff = cb.inv_phi - cn.inv_phi;
    float ubx = rho0 * diff * gux, uby = rho0 * diff * guy;
    const float Pn_b = -3.0f * W;  // adjoint of phi_n p_n
    float ipn_b = -rho0 * WA;       // adjoint of 1/phi_n
    const float ipb_b = rho0 * WA;  // adjoint of 1/phi_b
    // phi_n p_n (deviation) = 0.6 m1 - 0.4 rho0 |u|^2 / phi_n
    const float mb1 = 0.6f * Pn_b;
    ubx += -0.8f * rho0 * ux * cn.inv_phi * Pn_b;
    uby += -0.8f * rho0 * uy * cn.inv_phi * Pn_b;
    ipn_b += -0.4f * rho0 * usq * Pn_b;
    const VelBar vb = velocity_vjp(jx, jy, cn, P.ax, P.ay, P.inv_rho0, ubx, uby, 0.0f);
    nu[i * P.plane + on] += nbi + mb1 + ex * vb.jx + ey * vb.jy;
    if (i == 0) {
      // boundary cell: phi_b p_b and 1/phi_b
      g_phi[ob] += 3.0f * pb * W - cb.inv_phi * cb.inv_phi * ipb_b;
      float gl = 0.0f, gp = 0.0f;
      theta_bar(cn, vb.clin, vb.cnl, ipn_b, vb.phi, gl, gp);
      g_l[on] += gl;
      g_phi[on] += gp;
    }
  }
}

// J_W^T in place on nu: the wall nodes of the extrapolated sides.  A wall node b is overwritten by
//   W_b,i = f_eq,i(phi_b p_nb, u_w; phi_b) + z_nb,i - f_eq,i(phi_nb p_nb, u_nb; phi_nb),
// a function of the pre-boundary state z_nb of its inner neighbour, of phi_b and of theta at nb; so
// its adjoint is cleared and J^T lambda_b is added to nb.  A corner's nb is the diagonal node, which
// is also the nb of the wall nodes beside the corner: one group of eight lanes (lane i holding
// population i) per nb takes all the wall nodes that extrapolate from it, in a fixed order, so the
// sums are race-free and deterministic.  Groups: the nb of the bottom and top walls (row 1 / ny-2,
// with the corners and, when the x sides are extrapolated too, the side nodes of rows 1 and ny-2),
// then the nb of the left and right walls in the remaining rows.  Needs nx >= 4 on extrapolated
// x sides and ny >= 4 on extrapolated y sides (no nb on two sides at once, no nb that is a wall node).
struct WallGroups {
  int gy, gx, row0;  // groups per y side (bottom, top), per x side (left, right), first row of the x groups
};

__host__ __device__ inline WallGroups wall_groups(const StepParams& P) {
  WallGroups g;
  g.gy = P.bc_y == BC_NEE ? (P.bc_x == BC_PERIODIC ? P.nx : P.nx - 2) : 0;
  g.row0 = P.bc_y == BC_NEE ? 2 : 0;
  g.gx = P.bc_x == BC_NEE ? (P.bc_y == BC_NEE ? P.ny - 4 : P.ny) : 0;
  return g;
}

template <int PREC, bool HET>
__global__ void k_adj_wall(const StepParams P, const void* buf, WallGroups G, float* __restrict__ nu, float* __restrict__ g_l,
                           float* __restrict__ g_phi) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  int grp = t >> 3;
  const int i = t & 7;
  if (grp >= 2 * (G.gy + G.gx)) return;  // whole lane groups leave together
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  // the nb (xt, yt) of this group and the wall nodes (bx, by) on walls bw that extrapolate from it
  int xt, yt, n = 0;
  int bx[3], by[3], bw[3];
  if (grp < 2 * G.gy) {
    const int top = grp >= G.gy, g = grp - (top ? G.gy : 0);
    xt = P.bc_x == BC_PERIODIC ? g : g + 1;
    yt = top ? P.ny - 2 : 1;
    const int yw = top ? P.ny - 1 : 0, w = top ? 3 : 2;
    bx[n] = xt; by[n] = yw; bw[n++] = w;
    if (P.bc_x != BC_PERIODIC && xt == 1) { bx[n] = 0; by[n] = yw; bw[n++] = w; }
    if (P.bc_x != BC_PERIODIC && xt == P.nx - 2) { bx[n] = P.nx - 1; by[n] = yw; bw[n++] = w; }
    if (P.bc_x == BC_NEE && xt == 1) { bx[n] = 0; by[n] = yt; bw[n++] = 0; }
    if (P.bc_x == BC_NEE && xt == P.nx - 2) { bx[n] = P.nx - 1; by[n] = yt; bw[n++] = 1; }
  } else {
    grp -= 2 * G.gy;
    const int right = grp >= G.gx;
    yt = G.row0 + grp - (right ? G.gx : 0);
    xt = right ? P.nx - 2 : 1;
    bx[n] = right ? P.nx - 1 : 0; by[n] = yt; bw[n++] = right ? 1 : 0;
  }
  if (!dbg_check(P, xt >= 0 && xt < P.nx && yt >= 0 && yt < P.ny)) return;  // uniform over the lane group
  using T = typename Store<PREC>::T;
  const float ex = (float)ex_of(i), ey = (float)ey_of(i), wi = w_of(i);
  const float rho0 = P.rho0;
  // forward quantities at nb: u_nb (Eqs. 18-19), phi_nb p_nb (Eq. 20)
  const float zi = pull_one<PREC>(P, static_cast<const T*>(buf), xt, yt, i);
  const Coef cn = coef_at<HET>(P, xt, yt);
  const float jx = group8_sum(ex * zi, gm), jy = group8_sum(ey * zi, gm), m1 = group8_sum(zi, gm);
  float ux, uy, umag;
  velocity_from_j(jx, jy, cn, P.ax, P.ay, P.inv_rho0, ux, uy, umag);
  const float usq = ux * ux + uy * uy;
  const float Pn = P.p_rest + 0.6f * m1 - 0.4f * rho0 * usq * cn.inv_phi;  // phi_nb p_nb
  const float eun = ex * ux + ey * uy;
  // adjoints at nb, summed over the wall nodes: z_nb,i, phi_nb p_nb, 1/phi_nb, u_nb
  float zbar = 0.0f, Pn_b = 0.0f, ipn_b = 0.0f, ubx = 0.0f, uby = 0.0f;
  for (int k = 0; k < n; ++k) {
    if (!dbg_check(P, bx[k] >= 0 && bx[k] < P.nx && by[k] >= 0 && by[k] < P.ny)) continue;
    const int64_t ob = (int64_t)by[k] * P.pitch + bx[k];
    const float lam = nu[i * P.plane + ob];
    nu[i * P.plane + ob] = 0.0f;
    const Coef cb = coef_at<HET>(P, bx[k], by[k]);
    const float uwx = __ldg(P.uw + 2 * bw[k]), uwy = __ldg(P.uw + 2 * bw[k] + 1);
    const float euw = ex * uwx + ey * uwy;
    const float wl = wi * lam;
    const float W = group8_sum(wl, gm);
    const float WAw = group8_sum(wl * (4.5f * euw * euw - 1.5f * (uwx * uwx + uwy * uwy)), gm);
    const float WAn = group8_sum(wl * (4.5f * eun * eun - 1.5f * usq), gm);
    const float gux = group8_sum(wl * (3.0f * ex + (9.0f * eun * ex - 3.0f * ux) * cn.inv_phi), gm);
    const float guy = group8_sum(wl * (3.0f * ey + (9.0f * eun * ey - 3.0f * uy) * cn.inv_phi), gm);
    // phi_b p_nb = (1 + r) phi_nb p_nb with r = phi_b / phi_nb - 1
    const float r = cb.phi * cn.inv_phi - 1.0f;
    zbar += lam;
    Pn_b += 3.0f * r * W;
    const float r_b = 3.0f * W * Pn;
    ipn_b += r_b * cb.phi - rho0 * WAn;
    ubx += -rho0 * gux;
    uby += -rho0 * guy;
    if (i == 0) g_phi[ob] += r_b * cn.inv_phi - cb.inv_phi * cb.inv_phi * rho0 * WAw;  // phi_b through r and 1/phi_b
  }
  // phi_nb p_nb (deviation) = 0.6 m1 - 0.4 rho0 |u|^2 / phi_nb
  const float mb1 = 0.6f * Pn_b;
  ubx += -0.8f * rho0 * ux * cn.inv_phi * Pn_b;
  uby += -0.8f * rho0 * uy * cn.inv_phi * Pn_b;
  ipn_b += -0.4f * rho0 * usq * Pn_b;
  const VelBar vb = velocity_vjp(jx, jy, cn, P.ax, P.ay, P.inv_rho0, ubx, uby, 0.0f);
  const int64_t on = (int64_t)yt * P.pitch + xt;
  nu[i * P.plane + on] += zbar + mb1 + ex * vb.jx + ey * vb.jy;
  if (i == 0) {
    float gl = 0.0f, gp = 0.0f;
    theta_bar(cn, vb.clin, vb.cnl, ipn_b, vb.phi, gl, gp);
    g_l[on] += gl;
    g_phi[on] += gp;
  }
}

// nu(t) = J_C(z(t))^T P^T nu~(t+1), gradient += (dC/dtheta)^T P^T nu~(t+1); z(t) gathered from
// buf = b(t).  Generic form for one cell (frame cells): every boundary rule.
template <int PREC, bool HET>
__device__ void adj_cell(const StepParams& P, const void* buf, const AdjArgs& A, int x, int y) {
  // P^T: the slot (i, x) feeds the cell x + e_i, or the cell x itself through a wall
  float mu[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int tx = x + ex_of(i), ty = y + ey_of(i);
    if (P.bc_x != BC_WALL) tx = (tx + P.nx) % P.nx;
    if (P.bc_y != BC_WALL) ty = (ty + P.ny) % P.ny;
    if (tx >= 0 && tx < P.nx && ty >= 0 && ty < P.ny)
      mu[i] = A.nu_in[i * P.plane + (int64_t)ty * P.pitch + tx];
    else
      mu[i] = A.nu_in[opp_of(i) * P.plane + (int64_t)y * P.pitch + x];
  }
  float z[8];
  gather_z<PREC, HET>(P, buf, x, y, z);
  const Coef c = coef_at<HET>(P, x, y);
  float nu[8];
  float gl = 0.0f, gp = 0.0f;
  collide_vjp(z, c, P.ax, P.ay, P, mu, nu, gl, gp);
  const int64_t o = (int64_t)y * P.pitch + x;
#pragma unroll
  for (int i = 0; i < 8; ++i) A.nu_out[i * P.plane + o] = nu[i];
  A.g_l[o] += gl;
  A.g_phi[o] += gp;
}

// Work split of the adjoint step.  The frame is the forward kernel's (groups of four cells that
// touch a wall row or the first/last column), done one cell per thread; the rest of the lattice is
// split into pairs of cells, one pair per thread, which keeps half the forward kernel's live state
// per thread (the reverse-mode collision holds the forward state, the adjoint state and their
// partial adjoints) so that more warps stay resident.  Rows of P <= nt pairs are packed
// rows_per_item = nt / P to a work item, longer rows take gx = ceil(P / nt) items.
struct AdjTiling {
  int frame_blocks, pairs, gx, rows_per_item, frame_x1;  // frame_x1: first x of the last frame group
};

__host__ __device__ inline AdjTiling adj_tiling_of(int nx, int ny, int bc_y, int nt) {
  AdjTiling t;
  const Frame F = frame_of(nx, ny, bc_y, kCellsPerThread);
  t.frame_blocks = (int)(((int64_t)F.count * kCellsPerThread + nt - 1) / nt);
  t.pairs = (nx + 1) / 2;
  if (t.pairs <= nt) {
    t.gx = 1;
    t.rows_per_item = nt / t.pairs;
  } else {
    t.gx = (t.pairs + nt - 1) / nt;
    t.rows_per_item = 1;
  }
  t.frame_x1 = (F.groups_per_row - 1) * kCellsPerThread;
  return t;
}

inline int64_t adj_main_items(const AdjTiling& t, int ny) {
  return t.rows_per_item > 1 ? (int64_t)((ny + t.rows_per_item - 1) / t.rows_per_item) : (int64_t)t.gx * ny;
}

// Row and first cell of the pair of thread `tid` in main item b; false for a thread with no pair
// (it takes part in the loads and shuffles on a clamped row and stores nothing).
__device__ __forceinline__ bool adj_pair(const AdjTiling& t, int ny, int nt, int b, int tid, int& x0, int& y) {
  if (t.rows_per_item > 1) {
    const int r = tid / t.pairs;
    y = b * t.rows_per_item + r;
    x0 = (tid - r * t.pairs) * 2;
    const bool ok = r < t.rows_per_item && y < ny;
    if (!ok) y = ny - 1;
    return ok;
  }
  y = b / t.gx;
  x0 = ((b - y * t.gx) * nt + tid) * 2;
  return true;
}

// Work item of the adjoint step: frame items do the frame cell by cell; main items gather the
// forward state forwards and the adjoint state backwards (mu_i(x) = nu~_i(x + e_i)) for a pair
// of cells with shuffled halos, and skip the frame.
template <int PREC, bool HET, int NT>
__device__ __forceinline__ void adj_item(const StepParams& P, const void* buf, const AdjArgs& A, const AdjTiling& tl, int item) {
  using T = typename Store<PREC>::T;
  if (item < tl.frame_blocks) {  // one frame cell per thread
    const Frame F = frame_of(P.nx, P.ny, P.bc_y, kCellsPerThread);
    int x, y;
    if (frame_cell(F, P.ny, item * NT + (int)threadIdx.x, x, y) && x < P.nx && dbg_check(P, y >= 0 && y < P.ny))
      adj_cell<PREC, HET>(P, buf, A, x, y);
    return;
  }
  int x0, y;
  const bool has_pair = adj_pair(tl, P.ny, NT, item - tl.frame_blocks, (int)threadIdx.x, x0, y);
  const int lane = threadIdx.x & 31;
  int xl = x0 < P.pitch - 2 ? x0 : P.pitch - 2;
  const bool idx_ok = dbg_check(P, y >= 0 && y < P.ny && xl >= 0);
  if (!idx_ok) y = xl = 0;  // (debug builds) keep the loads and shuffles inside the buffers
  int ym = y - 1, yp = y + 1;
  ym = ym < 0 ? P.ny - 1 : ym;
  yp = yp >= P.ny ? 0 : yp;
  const int64_t pl = P.plane;
  const int64_t rm = (int64_t)ym * P.pitch, r0 = (int64_t)y * P.pitch, rp = (int64_t)yp * P.pitch;
  const T* __restrict__ src = static_cast<const T*>(buf);
  const float inv = P.inv_scale;
  // medium of the two cells, issued ahead of the state gathers
  float2 ph2, k2;
  if (HET) {
    ph2 = __ldg(reinterpret_cast<const float2*>(P.phi + r0 + xl));
    k2 = __ldg(reinterpret_cast<const float2*>(P.K + r0 + xl));
  }
  // forward state z(t): the pull of Eq. 15
  float z[8][2];
  gather2<PREC, 1>(src + 0 * pl + r0, xl, P.pitch, lane, inv, z[0]);
  gather2<PREC, 0>(src + 1 * pl + rm, xl, P.pitch, lane, inv, z[1]);
  gather2<PREC, -1>(src + 2 * pl + r0, xl, P.pitch, lane, inv, z[2]);
  gather2<PREC, 0>(src + 3 * pl + rp, xl, P.pitch, lane, inv, z[3]);
  gather2<PREC, 1>(src + 4 * pl + rm, xl, P.pitch, lane, inv, z[4]);
  gather2<PREC, -1>(src + 5 * pl + rm, xl, P.pitch, lane, inv, z[5]);
  gather2<PREC, -1>(src + 6 * pl + rp, xl, P.pitch, lane, inv, z[6]);
  gather2<PREC, 1>(src + 7 * pl + rp, xl, P.pitch, lane, inv, z[7]);
  // adjoint of the pull: mu_i(x) = nu~_i(x + e_i)
  const float* __restrict__ nu_in = A.nu_in;
  float mu[8][2];
  gather2<PREC_FP32, -1>(nu_in + 0 * pl + r0, xl, P.pitch, lane, 1.0f, mu[0]);  // e1 = ( 1, 0)
  gather2<PREC_FP32, 0>(nu_in + 1 * pl + rp, xl, P.pitch, lane, 1.0f, mu[1]);   // e2 = ( 0, 1)
  gather2<PREC_FP32, 1>(nu_in + 2 * pl + r0, xl, P.pitch, lane, 1.0f, mu[2]);   // e3 = (-1, 0)
  gather2<PREC_FP32, 0>(nu_in + 3 * pl + rm, xl, P.pitch, lane, 1.0f, mu[3]);   // e4 = ( 0,-1)
  gather2<PREC_FP32, -1>(nu_in + 4 * pl + rp, xl, P.pitch, lane, 1.0f, mu[4]);  // e5 = ( 1, 1)
  gather2<PREC_FP32, 1>(nu_in + 5 * pl + rp, xl, P.pitch, lane, 1.0f, mu[5]);   // e6 = (-1, 1)
  gather2<PREC_FP32, 1>(nu_in + 6 * pl + rm, xl, P.pitch, lane, 1.0f, mu[6]);   // e7 = (-1,-1)
  gather2<PREC_FP32, -1>(nu_in + 7 * pl + rm, xl, P.pitch, lane, 1.0f, mu[7]);  // e8 = ( 1,-1)
  const bool wall_row = (P.bc_y == BC_WALL || P.bc_y == BC_NEE) && (y == 0 || y == P.ny - 1);
  if (!has_pair || !idx_ok || wall_row || x0 < kCellsPerThread || x0 >= tl.frame_x1) return;
  float gl[2], gp[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    float zc[8], mc[8], nc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      zc[i] = z[i][c];
      mc[i] = mu[i][c];
    }
    const Coef cf = HET ? coef_of(P, c ? ph2.y : ph2.x, c ? k2.y : k2.x, P.sv ? __ldg(P.sv + r0 + x0 + c) : P.s_v) : coef_uniform(P);
    gl[c] = 0.0f;
    gp[c] = 0.0f;
    collide_vjp(zc, cf, P.ax, P.ay, P, mc, nc, gl[c], gp[c]);
#pragma unroll
    for (int i = 0; i < 8; ++i) z[i][c] = nc[i];
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) *reinterpret_cast<float2*>(A.nu_out + i * pl + r0 + x0) = make_float2(z[i][0], z[i][1]);
  float2* g2l = reinterpret_cast<float2*>(A.g_l + r0 + x0);
  float2* g2p = reinterpret_cast<float2*>(A.g_phi + r0 + x0);
  float2 a = *g2l, b = *g2p;
  a.x += gl[0]; a.y += gl[1];
  b.x += gp[0]; b.y += gp[1];
  *g2l = a;
  *g2p = b;
}

#ifndef LBM_ADJ_MIN_CTAS
#define LBM_ADJ_MIN_CTAS 7
#endif
template <int PREC, bool HET>
__global__ void __launch_bounds__(kStepThreads, LBM_ADJ_MIN_CTAS) k_adj_step(const StepParams P, const void* buf, AdjArgs A, AdjTiling tl) {
  adj_item<PREC, HET, kStepThreads>(P, buf, A, tl, blockIdx.x);
}

// Initial state: z(0) = f_eq(p0, u0; phi) (Eq. 22): dL/dphi += sum_i nu_i d f_eq,i / d phi.
template <bool HET>
__global__ void k_adj_init(const StepParams P, const float* __restrict__ nu, float* __restrict__ g_phi, float p0, float ux0, float uy0,
                           int phip_uniform) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= P.nx) return;
  const Coef c = coef_at<HET>(P, x, y);
  const float usq = ux0 * ux0 + uy0 * uy0;
  const float pterm = phip_uniform ? 0.0f : 3.0f * p0;
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float eu = (float)ex_of(i) * ux0 + (float)ey_of(i) * uy0;
    const float d = w_of(i) * (pterm - P.rho0 * (4.5f * eu * eu - 1.5f * usq) * c.inv_phi * c.inv_phi);
    s += d * nu[i * P.plane + (int64_t)y * P.pitch + x];
  }
  g_phi[(int64_t)y * P.pitch + x] += s;
}

// FP32 partial sums of the gradients into the FP64 totals, and the partial sums reset: run every
// few dozen steps, so that each FP32 sum holds a bounded number of per-step terms.
__global__ void k_adj_fold(float* __restrict__ l32, float* __restrict__ p32, double* __restrict__ l64, double* __restrict__ p64,
                           int64_t n) {
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    l64[k] += (double)l32[k];
    p64[k] += (double)p32[k];
    l32[k] = 0.0f;
    p32[k] = 0.0f;
  }
}

// --------------------------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------------------------
#define LBM_ADJ_DISPATCH(prec, het, CALL)                                        \
  do {                                                                            \
    if (prec == PREC_FP32) { if (het) { CALL(PREC_FP32, true); } else { CALL(PREC_FP32, false); } } \
    else if (prec == PREC_FP16) { if (het) { CALL(PREC_FP16, true); } else { CALL(PREC_FP16, false); } } \
    else { if (het) { CALL(PREC_BF16, true); } else { CALL(PREC_BF16, false); } } \
  } while (0)

cudaError_t launch_adj_seed(const StepParams& P, int prec, bool het, float* nu_out, float* g_l, float* g_phi, int kind,
                            const float* tux, const float* tuy, double* partial, int nblocks, double* loss_out, cudaStream_t s) {
  AdjArgs A{nullptr, nu_out, g_l, g_phi};
#define CALL_SEED(PR, H) k_adj_seed<PR, H><<<nblocks, 256, 0, s>>>(P, A, kind, tux, tuy, partial)
  LBM_ADJ_DISPATCH(prec, het, CALL_SEED);
#undef CALL_SEED
  k_adj_loss_total<<<1, 32, 0, s>>>(partial, nblocks, loss_out);
  return cudaGetLastError();
}

cudaError_t launch_adj_nee(const StepParams& P, int prec, bool het, const void* buf, float* nu, float* g_l, float* g_phi,
                           cudaStream_t s) {
  const int threads = 8 * (P.nx < 4 ? P.ny : 2 * P.ny);
  const int blocks = (threads + 127) / 128;
#define CALL_NEE(PR, H) k_adj_nee<PR, H><<<blocks, 128, 0, s>>>(P, buf, nu, g_l, g_phi)
  LBM_ADJ_DISPATCH(prec, het, CALL_NEE);
#undef CALL_NEE
  return cudaGetLastError();
}

cudaError_t launch_adj_wall(const StepParams& P, int prec, bool het, const void* buf, float* nu, float* g_l, float* g_phi,
                            cudaStream_t s) {
  const WallGroups G = wall_groups(P);
  const int threads = 8 * 2 * (G.gy + G.gx);
  if (threads == 0) return cudaSuccess;
  const int blocks = (threads + 127) / 128;
#define CALL_WALL(PR, H) k_adj_wall<PR, H><<<blocks, 128, 0, s>>>(P, buf, G, nu, g_l, g_phi)
  LBM_ADJ_DISPATCH(prec, het, CALL_WALL);
#undef CALL_WALL
  return cudaGetLastError();
}

cudaError_t launch_adj_step(const StepParams& P, int prec, bool het, const void* buf, const float* nu_in, float* nu_out, float* g_l,
                            float* g_phi, cudaStream_t s) {
  AdjArgs A{nu_in, nu_out, g_l, g_phi};
  const AdjTiling tl = adj_tiling_of(P.nx, P.ny, P.bc_y, kStepThreads);
  const unsigned blocks = (unsigned)((long long)tl.frame_blocks + adj_main_items(tl, P.ny));
#define CALL_ADJ(PR, H) k_adj_step<PR, H><<<blocks, kStepThreads, 0, s>>>(P, buf, A, tl)
  LBM_ADJ_DISPATCH(prec, het, CALL_ADJ);
#undef CALL_ADJ
  return cudaGetLastError();
}

cudaError_t launch_adj_init(const StepParams& P, bool het, const float* nu, float* g_phi, float p0, float ux0, float uy0,
                            int phip_uniform, cudaStream_t s) {
  dim3 grid((P.nx + 127) / 128, P.ny);
  if (het)
    k_adj_init<true><<<grid, 128, 0, s>>>(P, nu, g_phi, p0, ux0, uy0, phip_uniform);
  else
    k_adj_init<false><<<grid, 128, 0, s>>>(P, nu, g_phi, p0, ux0, uy0, phip_uniform);
  return cudaGetLastError();
}

cudaError_t launch_adj_fold(float* l32, float* p32, double* l64, double* p64, int64_t n, cudaStream_t s) {
  k_adj_fold<<<1216, 256, 0, s>>>(l32, p32, l64, p64, n);
  return cudaGetLastError();
}

}  // namespace lbm
