// Device-side building blocks of the porous D2Q8 MRT-LB step (Liu & He, arXiv 1311.7239) and of
// the D2Q5 temperature step (its Appendix B), for sm_103a.
//
// Storage: structure-of-arrays planes [q][ny][pitch].  Every plane holds the deviation of a
// post-collision population from the rest equilibrium, d_i = f_i - f_rest,i with
// f_rest,i = 3 w_i p_rest (Eq. 22 at u = 0, phi p = p_rest) for the flow and T0 / 5 (Eq. B.6 at
// u = 0, T = T0) for the temperature; FP16/BF16 planes scale d by 2^k.  The collision below works
// in those deviation variables throughout, which keeps FP32 arithmetic (and FP16 storage) far
// from the cancellation of subtracting two O(1) populations.
//
// One time step per cell (pull form of Eq. 15 followed by Eq. 14):
//   gather d_i(x - e_i) (bounce-back/periodic/pressure rules at the edges)
//   m = M d (Eq. 10, expanded), v, u (Eqs. 18-19), phi p (Eq. 20), F (Eq. 3), S (Eq. 16),
//   m+ = m - Lambda (m - m_eq) + (I - Lambda/2) S (Eqs. 11-14), d+ = M^-1 m+ (Eq. 8, expanded).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace lbm {

enum : int { PREC_FP32 = 0, PREC_FP16 = 1, PREC_BF16 = 2 };
enum : int { BC_PERIODIC = 0, BC_WALL = 1, BC_PRESSURE = 2, BC_NEE = 3 };

// Constants of the two-cell collision (collide_pair), derived on the host from the configuration.
// Moments there are taken of the stored (scaled) deviations s d, so every constant that turns a
// physical quantity into a moment increment carries the storage scale s (1 for FP32 and BF16).
struct PairConst {
  float inv_rho0s;             // 1 / (rho0 s)
  float nphip;                 // -(2/3) rho0 s                 (Eq. 20)
  float nse8, sq6, nsq12;      // -s_e / 8, s_q / 6, -s_q / 12   (Lambda times the diagonal of M^-1)
  float r3, r12;               // rho0 s / 3, rho0 s / 12        (rho0 F through M^-1)
  float hay;                   // a_y / 2
  float cq;                    // -s_v / 4
  // medium coefficients of the uniform medium (see PairCoef) and phi a / 2
  float u_inv_phi, u_l0, u_l0sq, u_l1, u_nclin, u_ncnl, u_c2, u_nR, u_cf7, u_cf8, u_hx, u_hy;
  // per-cell media (pair_coef_het): 0.1 (1 - s_e/2) rho0 s, rho0 s, a_x / 2
  float k_c2, k_rs, hax;
};

// Everything a step kernel needs, passed by value.
struct StepParams {
  const void* src;   // current post-collision planes (8)
  void* dst;         // next post-collision planes (8)
  const void* gsrc;  // temperature planes (5), thermal only
  void* gdst;
  const float* phi;  // per-cell porosity [ny][pitch], or nullptr for uniform
  const float* K;    // per-cell permeability [ny][pitch], or nullptr for uniform
  const float* sv;   // per-cell viscous rate s_v = 1/(1/2 + 3 J nu) [ny][pitch] (heterogeneous mode), or nullptr
  int nx, ny, pitch;
  int64_t plane;     // elements per plane = ny * pitch
  int bc_x, bc_y;
  int forch;
  int inplace;       // 1: one population buffer with in-place streaming (see ip_off), 0: A-B buffers
  int parity;        // in-place: parity of the next step (selects the slots it loads from)
  float rho0, inv_rho0, nu, s_e, s_q, s_v;
  float ax, ay;
  // uniform-medium coefficients
  float phi_u, inv_phi_u, c_lin_u, c_nl_u;
  const float* uw;    // wall velocities [4][2] in device memory: left, right, bottom, top
  float p_in, p_out;  // pressure columns
  float p_rest;       // phi p of the stored rest state
  float scale, inv_scale;  // storage scale 2^k (1 for FP32)
  // temperature
  float zeta1, zeta3, zeta4, inv_sigma, varpi, g_beta, T0;
  float Tw[4];
  int Tdir[4];        // 1 = wall temperature prescribed, 0 = adiabatic
  unsigned int* err;  // bit 0: non-finite velocity
  float* urec;        // in-place step: if set, the velocity of every cell's collision, dense [2][ny][nx]
  float* edge;        // in-place step with extrapolated sides: pre-collision states of the boundary nodes (see k_edge_ip)
  PairConst pc;
};

// Debug builds (-DLBM_DEBUG) check the index invariants of the kernels: a violation sets bit 2 of
// the error word, which the next synchronising call reports, and the access is skipped or clamped.
// Release builds compile the checks away.
__device__ __forceinline__ bool dbg_check(const StepParams& P, bool ok) {
#ifdef LBM_DEBUG
  if (!ok) atomicOr(P.err, 4u);
  return ok;
#else
  (void)P;
  (void)ok;
  return true;
#endif
}

// D2Q8 velocities of Eq. 7 and the weights w_i listed after Eq. 20 (w_1..4 = 1/9, w_5..8 = 1/36).
__device__ __forceinline__ int ex_of(int i) { return (i == 0 || i == 4 || i == 7) ? 1 : ((i == 2 || i == 5 || i == 6) ? -1 : 0); }
__device__ __forceinline__ int ey_of(int i) { return (i == 1 || i == 4 || i == 5) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0); }
__device__ __forceinline__ int opp_of(int i) { return i < 4 ? (i + 2) & 3 : 4 + ((i - 4 + 2) & 3); }
__device__ __forceinline__ float w_of(int i) { return i < 4 ? (1.0f / 9.0f) : (1.0f / 36.0f); }

// ---------------------------------------------------------------------------------------------
// storage codecs
// ---------------------------------------------------------------------------------------------
template <int PREC> struct Store;
// dec/enc and load4/store4 convert between stored and true deviations (the FP16 scale); decr,
// load4r and store4r move the stored values unchanged.
template <> struct Store<PREC_FP32> {
  using T = float;
  __device__ static __forceinline__ float decr(T v) { return v; }
  __device__ static __forceinline__ void load4r(const T* p, float o[4]) { load4(p, o, 1.0f); }
  __device__ static __forceinline__ void store4r(T* p, const float o[4]) { store4(p, o, 1.0f); }
  __device__ static __forceinline__ void store2r(T* p, float2 v) { *reinterpret_cast<float2*>(p) = v; }
  __device__ static __forceinline__ void load2(const T* p, float o[2], float) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    o[0] = v.x; o[1] = v.y;
  }
  __device__ static __forceinline__ float dec(T v, float) { return v; }
  __device__ static __forceinline__ T enc(float v, float) { return v; }
  __device__ static __forceinline__ void load4(const T* p, float o[4], float) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  }
  __device__ static __forceinline__ void store4(T* p, const float o[4], float) {
    *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
  }
};
template <> struct Store<PREC_FP16> {
  using T = __half;
  __device__ static __forceinline__ float decr(T v) { return __half2float(v); }
  __device__ static __forceinline__ void load4r(const T* p, float o[4]) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  __device__ static __forceinline__ void store4r(T* p, const float o[4]) {
    __half2 a = __floats2half2_rn(o[0], o[1]);
    __half2 b = __floats2half2_rn(o[2], o[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned int*>(&a);
    raw.y = *reinterpret_cast<unsigned int*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
  }
  __device__ static __forceinline__ void store2r(T* p, float2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v); }
  // a 32-bit word holding two stored values <-> the pair as float2 (no scale applied)
  __device__ static __forceinline__ float2 w2f(uint32_t w) { return __half22float2(*reinterpret_cast<const __half2*>(&w)); }
  __device__ static __forceinline__ uint32_t f2w(float2 v) {
    const __half2 h = __float22half2_rn(v);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static __forceinline__ uint32_t bits(T v) { return *reinterpret_cast<const unsigned short*>(&v); }
  __device__ static __forceinline__ void load2(const T* p, float o[2], float inv) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(p));
    o[0] = a.x * inv; o[1] = a.y * inv;
  }
  __device__ static __forceinline__ float dec(T v, float inv) { return __half2float(v) * inv; }
  __device__ static __forceinline__ T enc(float v, float sc) { return __float2half_rn(v * sc); }
  __device__ static __forceinline__ void load4(const T* p, float o[4], float inv) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
    o[0] = a.x * inv; o[1] = a.y * inv; o[2] = b.x * inv; o[3] = b.y * inv;
  }
  __device__ static __forceinline__ void store4(T* p, const float o[4], float sc) {
    __half2 a = __floats2half2_rn(o[0] * sc, o[1] * sc);
    __half2 b = __floats2half2_rn(o[2] * sc, o[3] * sc);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned int*>(&a);
    raw.y = *reinterpret_cast<unsigned int*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
  }
};
// BF16 keeps FP32's exponent range, so its deviations are stored unscaled (scale = 1).
template <> struct Store<PREC_BF16> {
  using T = __nv_bfloat16;
  __device__ static __forceinline__ float decr(T v) { return __bfloat162float(v); }
  __device__ static __forceinline__ void load4r(const T* p, float o[4]) { load4(p, o, 1.0f); }
  __device__ static __forceinline__ void store4r(T* p, const float o[4]) { store4(p, o, 1.0f); }
  __device__ static __forceinline__ void store2r(T* p, float2 v) { *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v); }
  // a BF16 value is the high half of its FP32 value
  __device__ static __forceinline__ float2 w2f(uint32_t w) { return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u)); }
  __device__ static __forceinline__ uint32_t f2w(float2 v) {
    const __nv_bfloat162 h = __float22bfloat162_rn(v);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
  __device__ static __forceinline__ uint32_t bits(T v) { return *reinterpret_cast<const unsigned short*>(&v); }
  __device__ static __forceinline__ void load2(const T* p, float o[2], float) {
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
    o[0] = a.x; o[1] = a.y;
  }
  __device__ static __forceinline__ float dec(T v, float) { return __bfloat162float(v); }
  __device__ static __forceinline__ T enc(float v, float) { return __float2bfloat16_rn(v); }
  __device__ static __forceinline__ void load4(const T* p, float o[4], float) {
    const uint2 raw = *reinterpret_cast<const uint2*>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&raw.y));
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
  __device__ static __forceinline__ void store4(T* p, const float o[4], float) {
    __nv_bfloat162 a = __floats2bfloat162_rn(o[0], o[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(o[2], o[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned int*>(&a);
    raw.y = *reinterpret_cast<unsigned int*>(&b);
    *reinterpret_cast<uint2*>(p) = raw;
  }
};

// ---------------------------------------------------------------------------------------------
// medium coefficients of one cell
// ---------------------------------------------------------------------------------------------
struct Coef {
  float phi, inv_phi;
  float s_v;    // viscous relaxation rate s7 = s8 (Eq. 13, Eq. 21 with upsilon_e = J upsilon)
  float c_lin;  // phi nu / K          (linear Darcy drag of Eq. 3)
  float c_nl;   // phi F_phi / sqrt(K)  (Forchheimer drag of Eq. 3; = 1.75 / sqrt(150 phi K) by Eq. 4)
};

// Reciprocal and square root through the SFU approximations (a few ulp), which the FP32 error
// budget of the method tolerates; sqrt of 0 is 0.
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }

__device__ __forceinline__ float f4_get(const float4& v, int c) { return c == 0 ? v.x : c == 1 ? v.y : c == 2 ? v.z : v.w; }

// Coefficients of a cell with porosity ph, permeability k and viscous rate sv (Eqs. 3-4, 13).
__device__ __forceinline__ Coef coef_of(const StepParams& P, float ph, float k, float sv) {
  Coef c;
  c.phi = ph;
  c.inv_phi = fast_rcp(ph);
  c.c_lin = ph * P.nu * fast_rcp(k);
  c.c_nl = P.forch ? 1.75f * rsqrtf(150.0f * ph * k) : 0.0f;
  c.s_v = sv;
  return c;
}

__device__ __forceinline__ Coef coef_uniform(const StepParams& P) {
  Coef c;
  c.phi = P.phi_u; c.inv_phi = P.inv_phi_u; c.c_lin = P.c_lin_u; c.c_nl = P.c_nl_u; c.s_v = P.s_v;
  return c;
}

template <bool HET>
__device__ __forceinline__ Coef coef_at(const StepParams& P, int x, int y) {
  if (!HET) return coef_uniform(P);
  const int64_t o = (int64_t)y * P.pitch + x;
  return coef_of(P, __ldg(P.phi + o), __ldg(P.K + o), P.sv ? __ldg(P.sv + o) : P.s_v);
}

// ---------------------------------------------------------------------------------------------
// macroscopic velocity and pressure deviation of a pre-collision cell (Eqs. 17-20)
// ---------------------------------------------------------------------------------------------
struct Macro {
  float dm1;       // sum of deviations (first moment of M applied to d)
  float ux, uy;    // velocity, Eq. 18
  float phip_dev;  // phi p - p_rest, Eq. 20
};

// Eqs. 18-19; also returns |u| = |v| / (l0 + sqrt(l0^2 + l1 |v|)) for the Forchheimer drag.
__device__ __forceinline__ void velocity_from_j(float jx, float jy, const Coef& c, float ax, float ay,
                                                float inv_rho0, float& ux, float& uy, float& umag) {
  // v = sum e f / rho0 + phi a / 2 ; l0 = (1 + phi nu / (2K)) / 2 ; l1 = phi F_phi / (2 sqrt K)
  const float vx = jx * inv_rho0 + 0.5f * c.phi * ax;
  const float vy = jy * inv_rho0 + 0.5f * c.phi * ay;
  const float l0 = 0.5f + 0.25f * c.c_lin;
  const float l1 = 0.5f * c.c_nl;
  const float vmag = fast_sqrt(vx * vx + vy * vy);
  // Eq. 18, the cancellation-free root of l1 |u|^2 + 2 l0 |u| - |v| = 0
  const float inv = fast_rcp(l0 + fast_sqrt(l0 * l0 + l1 * vmag));
  ux = vx * inv;
  uy = vy * inv;
  umag = vmag * inv;
}

// ---------------------------------------------------------------------------------------------
// collision of one cell in deviation variables, d[8] in (pre-collision), out (post-collision)
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void collide_d2q8(float d[8], const Coef& c, float ax, float ay, const StepParams& P,
                                             float& ux_out, float& uy_out, float& phip_out) {
  const float rho0 = P.rho0;
  // m = M d, Eq. 10 with shared partial sums
  const float a13 = d[0] + d[2], a24 = d[1] + d[3];
  const float d13 = d[0] - d[2], d24 = d[1] - d[3];
  const float s57 = d[4] + d[6], s68 = d[5] + d[7];
  const float t57 = d[4] - d[6], t68 = d[5] - d[7];
  const float diag = s57 + s68;
  const float m1 = a13 + a24 + diag;        // p      (deviation)
  const float m2 = -(a13 + a24) + diag;     // e      (deviation)
  const float dxs = t57 - t68;              // e_x-weighted diagonal sum
  const float dys = t57 + t68;              // e_y-weighted diagonal sum
  const float m3 = d13 + dxs;               // j_x  (q_x = -2 d13 + dxs enters k4 below)
  const float m5 = d24 + dys;               // j_y  (q_y = -2 d24 + dys enters k6 below)
  const float m7 = a13 - a24;               // p_xx
  const float m8 = s57 - s68;               // p_xy

  float ux, uy, umag;
  velocity_from_j(m3, m5, c, ax, ay, P.inv_rho0, ux, uy, umag);
  const float usq = ux * ux + uy * uy;
  // Eq. 20 with c_s^2 / (1 - w0) = 3/5 and s0 = -2|u|^2 / (3 phi): phi p = 3/5 (sum f - 2/3 rho0 |u|^2 / phi)
  const float phip_dev = 0.6f * (m1 - (2.0f / 3.0f) * rho0 * usq * c.inv_phi);
  // Eq. 3
  const float drag = c.c_lin + c.c_nl * umag;
  const float Fx = -drag * ux + c.phi * ax;
  const float Fy = -drag * uy + c.phi * ay;

  // Eqs. 11-14 as increments k = m+ - m = -Lambda (m - m_eq) + (I - Lambda/2) S.  m1 is conserved
  // (m1_eq = m1, S1 = 0); m3, m5 gain rho0 F for any s3, s5.  The q moments relax towards
  // -rho0 u, and m4 + rho0 u_x = (m4 + m3) + rho0 F_x / 2 by Eq. 17: that form avoids subtracting
  // two O(u) numbers.  Adding the increments to the pulled populations (instead of rebuilding
  // them from m+) keeps FP32 rounding at about one unit of d per step.
  const float s_e = P.s_e, s_q = P.s_q, s_v = c.s_v;
  const float rFx = rho0 * Fx, rFy = rho0 * Fy;
  const float S2 = rho0 * 0.8f * (ux * Fx + uy * Fy) * c.inv_phi;
  const float k2 = -s_e * (m2 + phip_dev) + (1.0f - 0.5f * s_e) * S2;  // e_eq = -phi p
  const float k3 = rFx;
  const float k4 = -s_q * ((2.0f * dxs - d13) + 0.5f * rFx) - (1.0f - 0.5f * s_q) * rFx;
  const float k5 = rFy;
  const float k6 = -s_q * ((2.0f * dys - d24) + 0.5f * rFy) - (1.0f - 0.5f * s_q) * rFy;
  const float hv = 1.0f - 0.5f * s_v;
  const float k7 = -s_v * (m7 - rho0 * (ux * ux - uy * uy) * c.inv_phi) + hv * 2.0f * rho0 * (ux * Fx - uy * Fy) * c.inv_phi;
  const float k8 = -s_v * (m8 - rho0 * ux * uy * c.inv_phi) + hv * rho0 * (ux * Fy + uy * Fx) * c.inv_phi;

  // d+ = d + M^-1 k, M^-1 = M^T diag(1/8, 1/8, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4), k1 = 0
  const float q2 = k2 * 0.125f;
  const float q3 = k3 * (1.0f / 6.0f), q4 = k4 * (1.0f / 12.0f);
  const float q5 = k5 * (1.0f / 6.0f), q6 = k6 * (1.0f / 12.0f);
  const float q7 = k7 * 0.25f, q8 = k8 * 0.25f;
  const float X = q3 - 2.0f * q4, Y = q5 - 2.0f * q6;
  const float Px = q3 + q4, Py = q5 + q6;
  d[0] += (X + q7) - q2;
  d[1] += (Y - q7) - q2;
  d[2] += (q7 - X) - q2;
  d[3] += (-Y - q7) - q2;
  d[4] += (Px + Py + q8) + q2;
  d[5] += (Py - Px - q8) + q2;
  d[6] += (q8 - Px - Py) + q2;
  d[7] += (Px - Py - q8) + q2;
  ux_out = ux;
  uy_out = uy;
  phip_out = phip_dev;
}

// ---------------------------------------------------------------------------------------------
// The same collision for two cells at once, on the packed FP32 pairs of sm_100+ (FADD2, FMUL2,
// FFMA2: one instruction for both cells, each lane rounded as the scalar operation).  d holds the
// stored deviations s d of the two cells (s: storage scale), so the scale is folded into the
// constants instead of being applied on every load and store; u is returned in lattice units.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Medium coefficients of a cell pair (Eqs. 3-4, 13, 18), scaled as PairConst says (uniform medium:
// the same for both cells, from the host).
struct PairCoef {
  float2 inv_phi;     // 1 / phi
  float2 l0, l0sq;    // l0 = 1/2 + c_lin / 4 and l0^2 (Eq. 18)
  float2 l1;          // l1 = c_nl / 2
  float2 nclin, ncnl; // -c_lin = -phi nu / K, -c_nl = -1.75 / sqrt(150 phi K)
  float2 c2;          // 0.1 (1 - s_e/2) rho0 s / phi     (S2 / 8 = c2 (u . F))
  float2 cq;          // -s_v / 4
  float2 nR;          // -rho0 s / phi
  float2 cf7, cf8;    // (1 - s_v/2) rho0 s / (2 phi), / (4 phi)
};

__device__ __forceinline__ PairCoef pair_coef_uniform(const PairConst& K) {
  PairCoef c;
  c.inv_phi = f2(K.u_inv_phi); c.l0 = f2(K.u_l0); c.l0sq = f2(K.u_l0sq); c.l1 = f2(K.u_l1);
  c.nclin = f2(K.u_nclin); c.ncnl = f2(K.u_ncnl); c.c2 = f2(K.u_c2); c.cq = f2(K.cq); c.nR = f2(K.u_nR);
  c.cf7 = f2(K.u_cf7); c.cf8 = f2(K.u_cf8);
  return c;
}

// The same for a pair of cells of a per-cell medium: porosity ph, permeability k and viscous rate
// sv of the two cells (Eqs. 3-4, 13, 18, as coef_of); hx, hy receive phi a / 2.
__device__ __forceinline__ PairCoef pair_coef_het(const StepParams& P, float2 ph, float2 k, float2 sv, float2& hx, float2& hy) {
  const PairConst& K = P.pc;
  PairCoef c;
  c.inv_phi = make_float2(fast_rcp(ph.x), fast_rcp(ph.y));
  const float2 clin = mul2(mul2(ph, f2(P.nu)), make_float2(fast_rcp(k.x), fast_rcp(k.y)));  // phi nu / K
  const float2 cnl = P.forch ? make_float2(1.75f * rsqrtf(150.0f * ph.x * k.x), 1.75f * rsqrtf(150.0f * ph.y * k.y)) : f2(0.0f);
  c.l0 = fma2(f2(0.25f), clin, f2(0.5f));
  c.l0sq = mul2(c.l0, c.l0);
  c.l1 = mul2(f2(0.5f), cnl);
  c.nclin = neg2(clin);
  c.ncnl = neg2(cnl);
  const float2 rs_phi = mul2(f2(K.k_rs), c.inv_phi);
  c.c2 = mul2(f2(K.k_c2), c.inv_phi);
  c.cq = mul2(f2(-0.25f), sv);
  c.nR = neg2(rs_phi);
  const float2 hvr = mul2(fma2(f2(-0.5f), sv, f2(1.0f)), rs_phi);  // (1 - s_v/2) rho0 s / phi
  c.cf7 = mul2(f2(0.5f), hvr);
  c.cf8 = mul2(f2(0.25f), hvr);
  hx = mul2(f2(K.hax), ph);
  hy = mul2(f2(K.hay), ph);
  return c;
}

// hx, hy: phi a / 2 of the two cells.  d: in, stored pre-collision deviations; out, post-collision.
__device__ __forceinline__ void collide_pair(float2 d[8], const PairCoef& c, float2 hx, float2 hy, const PairConst& K, float2& ux,
                                             float2& uy) {
  // m = M d, Eq. 10 (as collide_d2q8)
  const float2 a13 = add2(d[0], d[2]), a24 = add2(d[1], d[3]);
  const float2 d13 = sub2(d[0], d[2]), d24 = sub2(d[1], d[3]);
  const float2 s57 = add2(d[4], d[6]), s68 = add2(d[5], d[7]);
  const float2 t57 = sub2(d[4], d[6]), t68 = sub2(d[5], d[7]);
  const float2 diag = add2(s57, s68), A = add2(a13, a24);
  const float2 m1 = add2(A, diag), m2 = sub2(diag, A);
  const float2 dxs = sub2(t57, t68), dys = add2(t57, t68);
  const float2 m3 = add2(d13, dxs), m5 = add2(d24, dys);
  const float2 m7 = sub2(a13, a24), m8 = sub2(s57, s68);

  // Eqs. 18-19: v = j / rho0 + phi a / 2, |u| = |v| / (l0 + sqrt(l0^2 + l1 |v|))
  const float2 vx = fma2(m3, f2(K.inv_rho0s), hx), vy = fma2(m5, f2(K.inv_rho0s), hy);
  const float2 vsq = fma2(vx, vx, mul2(vy, vy));
  const float2 vmag = mul2(vsq, make_float2(vsq.x > 0.0f ? rsqrtf(vsq.x) : 0.0f, vsq.y > 0.0f ? rsqrtf(vsq.y) : 0.0f));
  const float2 t = fma2(c.l1, vmag, c.l0sq);  // >= l0^2 >= 1/4
  const float2 den = add2(c.l0, mul2(t, make_float2(rsqrtf(t.x), rsqrtf(t.y))));
  const float2 inv = make_float2(fast_rcp(den.x), fast_rcp(den.y));
  ux = mul2(vx, inv);
  uy = mul2(vy, inv);
  const float2 umag = mul2(vmag, inv);
  // Eq. 20: phi p - p_rest = 3/5 (m1 - 2/3 rho0 |u|^2 / phi)   (times s)
  const float2 phip = mul2(f2(0.6f), fma2(f2(K.nphip), mul2(fma2(ux, ux, mul2(uy, uy)), c.inv_phi), m1));
  // Eq. 3: F = -(c_lin + c_nl |u|) u + phi a
  const float2 nd = fma2(c.ncnl, umag, c.nclin);
  const float2 Fx = fma2(nd, ux, add2(hx, hx)), Fy = fma2(nd, uy, add2(hy, hy));

  // increments k = m+ - m (Eqs. 11-14, as collide_d2q8) times the diagonal of M^-1:
  //   q2 = k2/8, X = k3/6 - k4/6 = rho0 F_x / 3 + s_q (m4 + m3) / 6, P_x = k3/6 + k4/12 =
  //   rho0 F_x / 12 - s_q (m4 + m3) / 12 (k4 = -s_q (m4 + m3) - rho0 F_x), q7 = k7/4, q8 = k8/4
  const float2 pxF = mul2(ux, Fx), pyF = mul2(uy, Fy);
  const float2 q2 = fma2(f2(K.nse8), add2(m2, phip), mul2(c.c2, add2(pxF, pyF)));
  const float2 gx = fma2(f2(2.0f), dxs, neg2(d13)), gy = fma2(f2(2.0f), dys, neg2(d24));  // m4 + m3, m6 + m5
  const float2 X = fma2(f2(K.sq6), gx, mul2(f2(K.r3), Fx)), Y = fma2(f2(K.sq6), gy, mul2(f2(K.r3), Fy));
  const float2 Px = fma2(f2(K.nsq12), gx, mul2(f2(K.r12), Fx)), Py = fma2(f2(K.nsq12), gy, mul2(f2(K.r12), Fy));
  const float2 q7 = fma2(c.cq, fma2(c.nR, fma2(ux, ux, neg2(mul2(uy, uy))), m7), mul2(c.cf7, sub2(pxF, pyF)));
  const float2 q8 = fma2(c.cq, fma2(c.nR, mul2(ux, uy), m8), mul2(c.cf8, fma2(ux, Fy, mul2(uy, Fx))));

  // d+ = d + M^-1 k (as collide_d2q8, with shared partial sums)
  const float2 B = sub2(q7, q2), Cn = add2(q7, q2);
  d[0] = add2(d[0], add2(B, X));
  d[2] = add2(d[2], sub2(B, X));
  d[1] = add2(d[1], sub2(Y, Cn));
  d[3] = sub2(d[3], add2(Y, Cn));
  const float2 G = add2(q8, q2), H = sub2(q2, q8), PP = add2(Px, Py), PM = sub2(Px, Py);
  d[4] = add2(d[4], add2(PP, G));
  d[6] = add2(d[6], sub2(G, PP));
  d[5] = add2(d[5], sub2(H, PM));
  d[7] = add2(d[7], add2(H, PM));
}

// macroscopic quantities only (no collision), for read-out kernels
__device__ __forceinline__ Macro macro_d2q8(const float d[8], const Coef& c, float ax, float ay, float rho0) {
  Macro r;
  const float m1 = d[0] + d[1] + d[2] + d[3] + d[4] + d[5] + d[6] + d[7];
  const float jx = (d[0] - d[2]) + (d[4] - d[5] - d[6] + d[7]);
  const float jy = (d[1] - d[3]) + (d[4] + d[5] - d[6] - d[7]);
  float umag;
  velocity_from_j(jx, jy, c, ax, ay, fast_rcp(rho0), r.ux, r.uy, umag);
  r.dm1 = m1;
  r.phip_dev = 0.6f * (m1 - (2.0f / 3.0f) * rho0 * (r.ux * r.ux + r.uy * r.uy) * c.inv_phi);
  return r;
}

// Equilibrium deviation f_eq,i(p, u; phi) - f_rest,i (Eq. 22 with rho0), phip_dev = phi p - p_rest.
__device__ __forceinline__ void feq_dev_d2q8(float phip_dev, float ux, float uy, float inv_phi, float rho0, float out[8]) {
  const float usq15 = 1.5f * (ux * ux + uy * uy) * inv_phi;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float eu = (float)ex_of(i) * ux + (float)ey_of(i) * uy;
    out[i] = w_of(i) * (3.0f * phip_dev + rho0 * (3.0f * eu + 4.5f * eu * eu * inv_phi - usq15));
  }
}

// ---------------------------------------------------------------------------------------------
// D2Q5 temperature collision in deviation variables (Eq. B.2 with n_eq of Eq. B.6)
// g[5]: deviations from T0/5, in (pre-collision) and out (post-collision); returns T.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float collide_d2q5(float g[5], float ux, float uy, const StepParams& P) {
  // n = N g, Eq. B.4
  const float n0 = g[0] + g[1] + g[2] + g[3] + g[4];
  const float n1 = g[1] - g[3];
  const float n2 = g[2] - g[4];
  const float side = g[1] + g[2] + g[3] + g[4];
  const float n3 = side - 4.0f * g[0];
  const float n4 = g[1] - g[2] + g[3] - g[4];
  const float T = P.T0 + n0;
  // increments n+ - n (n0 conserved), then g+ = g + N^-1 (n+ - n) with
  // N^-1 = N^T diag(1/5, 1/2, 1/2, 1/20, 1/4)
  const float r1 = -0.5f * P.zeta1 * (n1 - ux * T * P.inv_sigma);
  const float r2 = -0.5f * P.zeta1 * (n2 - uy * T * P.inv_sigma);
  const float r3 = -0.05f * P.zeta3 * (n3 - P.varpi * T);
  const float r4 = -0.25f * P.zeta4 * n4;
  g[0] += -4.0f * r3;
  g[1] += (r1 + r3) + r4;
  g[2] += (r2 + r3) - r4;
  g[3] += (r3 - r1) + r4;
  g[4] += (r3 - r2) - r4;
  return T;
}

// The same for two cells at once on packed FP32 pairs; g holds the stored deviations s g (s: the
// storage scale), u is in lattice units.  T = T0 + n0 / s is carried as s T = s T0 + n0.
__device__ __forceinline__ void collide_d2q5_pair(float2 g[5], float2 ux, float2 uy, const StepParams& P) {
  const float2 n0 = add2(add2(add2(g[0], g[1]), add2(g[2], g[3])), g[4]);
  const float2 n1 = sub2(g[1], g[3]), n2 = sub2(g[2], g[4]);
  const float2 side = add2(add2(g[1], g[2]), add2(g[3], g[4]));
  const float2 n3 = fma2(f2(-4.0f), g[0], side);
  const float2 n4 = sub2(add2(g[1], g[3]), add2(g[2], g[4]));
  const float2 sT = add2(f2(P.scale * P.T0), n0);  // s T
  const float2 q = mul2(sT, f2(P.inv_sigma));
  // increments n+ - n (n0 conserved) times the diagonal of N^-1 (as collide_d2q5)
  const float2 r1 = mul2(f2(-0.5f * P.zeta1), fma2(neg2(ux), q, n1));
  const float2 r2 = mul2(f2(-0.5f * P.zeta1), fma2(neg2(uy), q, n2));
  const float2 r3 = mul2(f2(-0.05f * P.zeta3), fma2(f2(-P.varpi), sT, n3));
  const float2 r4 = mul2(f2(-0.25f * P.zeta4), n4);
  const float2 a = add2(r3, r4), b = sub2(r3, r4);
  g[0] = fma2(f2(-4.0f), r3, g[0]);
  g[1] = add2(g[1], add2(r1, a));
  g[2] = add2(g[2], add2(r2, b));
  g[3] = add2(g[3], sub2(a, r1));
  g[4] = add2(g[4], sub2(b, r2));
}

// D2Q5 velocities of Eq. B.3 (0 rest, 1..4 as D2Q8's first four)
__device__ __forceinline__ int ex5(int i) { return i == 1 ? 1 : (i == 3 ? -1 : 0); }
__device__ __forceinline__ int ey5(int i) { return i == 2 ? 1 : (i == 4 ? -1 : 0); }
__device__ __forceinline__ int opp5(int i) { return i == 0 ? 0 : 1 + ((i - 1 + 2) & 3); }

// ---------------------------------------------------------------------------------------------
// generic pull of one population with every edge rule (used on edge cells and read-outs)
// ---------------------------------------------------------------------------------------------
// Wall that owns a link whose source (sx, sy) lies outside: y sides first (corners included).
__device__ __forceinline__ int wall_of(int sx, int sy, int ny) {
  if (sy < 0) return 2;
  if (sy >= ny) return 3;
  return sx < 0 ? 0 : 1;
}

// ---------------------------------------------------------------------------------------------
// In-place streaming: one population buffer.  Of each pair of opposite velocities the member with
// e_x > 0, or e_x = 0 and e_y > 0 (e1, e2, e5, e8), is "positive".  At parity par a cell c reads
// population i from plane (par ? i : opp(i)) at c itself when i is positive and at c - e_i
// otherwise, and writes its post-collision population j where the cell c + e_j reads j at the
// next parity.  The slots a cell writes are then exactly the slots it read (each receives the
// population opposite to the one read from it), so the two halves of Eq. 15 share one buffer
// without races and the buffer alternates between two layouts.  Populations that leave through a
// wall are parked in ghost slots (rows -1 and ny, column nx; never updated as cells) until the
// same cell reads them back as its bounce-back (Eq. 15 at a wall).  Ghost rows -1 and ny are rows of
// the planes; the ghost column lives after the last plane, q columns of ny + 2 slots (so that a
// lattice width that is a multiple of the row pitch needs no wider rows).  Extrapolated sides (wall
// nodes, pressure columns) keep the slot rules of a halfway wall; their boundary nodes' states are
// computed before each step (k_edge_ip), since they read a neighbour that the step overwrites.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ bool ip_positive(int i) { return i == 0 || i == 1 || i == 4 || i == 7; }

__device__ __forceinline__ int wrap_periodic(int v, int n, bool periodic) {
  return periodic ? (v < 0 ? v + n : (v >= n ? v - n : v)) : v;
}

// element offset (from row 0 of plane 0) of slot (plane, cx, cy) of a buffer of q planes
__device__ __forceinline__ int64_t ip_slot(const StepParams& P, int q, int plane, int cx, int cy) {
  if (cx >= P.nx) return (int64_t)q * P.plane - P.pitch + (int64_t)plane * (P.ny + 2) + (cy + 1);  // ghost column
  return (int64_t)plane * P.plane + (int64_t)cy * P.pitch + cx;
}

// element offset of the slot from which cell (cx, cy) (a lattice or ghost cell) reads population
// i at parity par
__device__ __forceinline__ int64_t ip_off(const StepParams& P, int cx, int cy, int i, int par) {
  if (!ip_positive(i)) {
    cx -= ex_of(i);
    cy -= ey_of(i);
  }
  cx = wrap_periodic(cx, P.nx, P.bc_x == BC_PERIODIC);
  cy = wrap_periodic(cy, P.ny, P.bc_y == BC_PERIODIC);
  dbg_check(P, cx >= 0 && cx <= P.nx && cy >= -1 && cy <= P.ny);
  return ip_slot(P, 8, par ? i : opp_of(i), cx, cy);
}

// the same for the D2Q5 temperature populations (positive: 1 and 2; the rest population stays)
__device__ __forceinline__ int64_t ip_off5(const StepParams& P, int cx, int cy, int i, int par) {
  if (i == 3 || i == 4) {
    cx -= ex5(i);
    cy -= ey5(i);
  }
  cx = wrap_periodic(cx, P.nx, P.bc_x == BC_PERIODIC);
  cy = wrap_periodic(cy, P.ny, P.bc_y == BC_PERIODIC);
  dbg_check(P, cx >= 0 && cx <= P.nx && cy >= -1 && cy <= P.ny);
  return ip_slot(P, 5, i == 0 ? 0 : (par ? i : opp5(i)), cx, cy);
}

// Source of the pull of population i into cell (x, y) at the current parity: the slot the cell
// reads (wall = -1), or, where x - e_i lies beyond a wall, the slot in which the cell parked its
// own post-collision population opp(i) (wall = the wall's index).
__device__ __forceinline__ int64_t ip_source(const StepParams& P, int x, int y, int i, int& wall) {
  int sx = x - ex_of(i), sy = y - ey_of(i);
  sx = wrap_periodic(sx, P.nx, P.bc_x == BC_PERIODIC);
  sy = wrap_periodic(sy, P.ny, P.bc_y == BC_PERIODIC);
  if (sx >= 0 && sx < P.nx && sy >= 0 && sy < P.ny) {
    wall = -1;
    return ip_off(P, x, y, i, P.parity);
  }
  wall = wall_of(sx, sy, P.ny);
  return ip_off(P, sx, sy, opp_of(i), P.parity);
}

__device__ __forceinline__ int64_t ip_source5(const StepParams& P, int x, int y, int i, int& wall) {
  int sx = x - ex5(i), sy = y - ey5(i);
  sx = wrap_periodic(sx, P.nx, P.bc_x == BC_PERIODIC);
  sy = wrap_periodic(sy, P.ny, P.bc_y == BC_PERIODIC);
  if (sx >= 0 && sx < P.nx && sy >= 0 && sy < P.ny) {
    wall = -1;
    return ip_off5(P, x, y, i, P.parity);
  }
  wall = wall_of(sx, sy, P.ny);
  return ip_off5(P, sx, sy, opp5(i), P.parity);
}

// momentum correction of the moving-wall bounce-back, 2 w_i rho0 (e_i . u_w) / c_s^2
__device__ __forceinline__ float wall_term(const StepParams& P, int i, int w) {
  return 6.0f * w_of(i) * P.rho0 * ((float)ex_of(i) * __ldg(P.uw + 2 * w) + (float)ey_of(i) * __ldg(P.uw + 2 * w + 1));
}

template <int PREC>
__device__ __forceinline__ float pull_one(const StepParams& P, const typename Store<PREC>::T* src, int x, int y, int i) {
  using S = Store<PREC>;
  if (!dbg_check(P, x >= 0 && x < P.pitch && y >= 0 && y < P.ny)) return 0.0f;
  if (P.inplace) {
    int w;
    const float v = S::dec(src[ip_source(P, x, y, i, w)], P.inv_scale);
    return w < 0 ? v : v + wall_term(P, i, w);
  }
  int sx = x - ex_of(i), sy = y - ey_of(i);
  if (P.bc_x != BC_WALL) sx = (sx + P.nx) % P.nx;
  if (P.bc_y != BC_WALL) sy = (sy + P.ny) % P.ny;
  if (sx >= 0 && sx < P.nx && sy >= 0 && sy < P.ny)
    return S::dec(src[(int64_t)i * P.plane + (int64_t)sy * P.pitch + sx], P.inv_scale);
  // halfway bounce-back: f_i(x) = f+_opp(i)(x) + 2 w_i rho0 (e_i . u_w) / c_s^2
  const int w = wall_of(sx, sy, P.ny);
  const int o = opp_of(i);
  const float own = S::dec(src[(int64_t)o * P.plane + (int64_t)y * P.pitch + x], P.inv_scale);
  return own + 6.0f * w_of(i) * P.rho0 * ((float)ex_of(i) * __ldg(P.uw + 2 * w) + (float)ey_of(i) * __ldg(P.uw + 2 * w + 1));
}

template <int PREC>
__device__ __forceinline__ void pull_cell(const StepParams& P, const typename Store<PREC>::T* src, int x, int y, float d[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = pull_one<PREC>(P, src, x, y, i);
}

// temperature: anti-bounce-back at walls with a prescribed temperature, bounce-back otherwise
template <int PREC>
__device__ __forceinline__ float pull_one_g(const StepParams& P, const typename Store<PREC>::T* src, int x, int y, int i) {
  using S = Store<PREC>;
  if (!dbg_check(P, x >= 0 && x < P.pitch && y >= 0 && y < P.ny)) return 0.0f;
  if (P.inplace) {
    int w;
    const float v = S::dec(src[ip_source5(P, x, y, i, w)], P.inv_scale);
    return (w < 0 || !P.Tdir[w]) ? v : (-v + 0.4f * (P.Tw[w] - P.T0));
  }
  if (i == 0) return S::dec(src[(int64_t)y * P.pitch + x], P.inv_scale);
  int sx = x - ex5(i), sy = y - ey5(i);
  if (P.bc_x != BC_WALL) sx = (sx + P.nx) % P.nx;
  if (P.bc_y != BC_WALL) sy = (sy + P.ny) % P.ny;
  if (sx >= 0 && sx < P.nx && sy >= 0 && sy < P.ny)
    return S::dec(src[(int64_t)i * P.plane + (int64_t)sy * P.pitch + sx], P.inv_scale);
  const int w = wall_of(sx, sy, P.ny);
  const float own = S::dec(src[(int64_t)opp5(i) * P.plane + (int64_t)y * P.pitch + x], P.inv_scale);
  // deviation form of g_i = -g+_opp + 2 T_w / 5 (reference T0 / 5): d_i = -d+_opp + 2 (T_w - T0) / 5
  return P.Tdir[w] ? (-own + 0.4f * (P.Tw[w] - P.T0)) : own;
}

template <int PREC>
__device__ __forceinline__ void pull_cell_g(const StepParams& P, const typename Store<PREC>::T* src, int x, int y, float g[5]) {
#pragma unroll
  for (int i = 0; i < 5; ++i) g[i] = pull_one_g<PREC>(P, src, x, y, i);
}

// Non-equilibrium extrapolation of a pressure column: replaces d of the cell (xb, y) by
// f_eq(p_b, u_nb; phi_b) + f_nb - f_eq(p_nb, u_nb; phi_nb) with nb = (xb +- 1, y), in deviations.
// (dn: the pulled state of nb)
template <bool HET>
__device__ __forceinline__ void pressure_column_from(const StepParams& P, const float dn[8], int xb, int y, float d[8]) {
  const int xn = xb == 0 ? 1 : P.nx - 2;
  const float pb = xb == 0 ? P.p_in : P.p_out;
  const Coef cn = coef_at<HET>(P, xn, y);
  const Coef cb = coef_at<HET>(P, xb, y);
  const Macro mn = macro_d2q8(dn, cn, P.ax, P.ay, P.rho0);
  float eb[8], en[8];
  feq_dev_d2q8(cb.phi * pb - P.p_rest, mn.ux, mn.uy, cb.inv_phi, P.rho0, eb);
  feq_dev_d2q8(mn.phip_dev, mn.ux, mn.uy, cn.inv_phi, P.rho0, en);
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = eb[i] + dn[i] - en[i];
}

template <int PREC, bool HET>
__device__ __forceinline__ void pressure_column(const StepParams& P, const typename Store<PREC>::T* src, int xb, int y, float d[8]) {
  float dn[8];
  pull_cell<PREC>(P, src, xb == 0 ? 1 : P.nx - 2, y, dn);
  pressure_column_from<HET>(P, dn, xb, y, d);
}

// Wall node of a side with non-equilibrium extrapolation (BC_NEE, the paper's wall treatment of
// Sec. 3): true for (x, y) on such a wall, with nb = (xn, yn) one step inward along the wall
// normal and w the wall (0 left, 1 right, 2 bottom, 3 top).  Bottom/top walls own the corners,
// whose nb is the diagonal node when the x sides are not periodic.
__device__ __forceinline__ bool nee_node(const StepParams& P, int x, int y, int& xn, int& yn, int& w) {
  if (P.bc_y == BC_NEE && (y == 0 || y == P.ny - 1)) {
    yn = y == 0 ? 1 : P.ny - 2;
    w = y == 0 ? 2 : 3;
    xn = (P.bc_x != BC_PERIODIC && (x == 0 || x == P.nx - 1)) ? (x == 0 ? 1 : P.nx - 2) : x;
    return true;
  }
  if (P.bc_x == BC_NEE && (x == 0 || x == P.nx - 1)) {
    xn = x == 0 ? 1 : P.nx - 2;
    yn = y;
    w = x == 0 ? 0 : 1;
    return true;
  }
  return false;
}

// d of a wall node: f_eq(p_nb, u_w; phi_b) + f_nb - f_eq(p_nb, u_nb; phi_nb) (pressure extrapolated
// with zero normal gradient), in deviations; ay_nb is a_y at nb (with its buoyancy in a thermal
// context), u_nb is returned; dn is the pulled state of nb.
template <bool HET>
__device__ __forceinline__ void wall_node_from(const StepParams& P, const float dn[8], int x, int y, int xn, int yn, int w, float ay_nb,
                                               float d[8], float& ux_nb, float& uy_nb) {
  const Coef cn = coef_at<HET>(P, xn, yn);
  const Coef cb = coef_at<HET>(P, x, y);
  const Macro mn = macro_d2q8(dn, cn, P.ax, ay_nb, P.rho0);
  ux_nb = mn.ux;
  uy_nb = mn.uy;
  // phi_b p_nb - p_rest = phi_nb p_nb - p_rest + (phi_b / phi_nb - 1) phi_nb p_nb, kept in deviations
  // (exact for phi_b = phi_nb; forming p_nb itself would add p_rest to a small deviation)
  const float dr = (cb.phi - cn.phi) * cn.inv_phi;
  const float phip_b = mn.phip_dev + dr * (mn.phip_dev + P.p_rest);
  float eb[8], en[8];
  feq_dev_d2q8(phip_b, __ldg(P.uw + 2 * w), __ldg(P.uw + 2 * w + 1), cb.inv_phi, P.rho0, eb);
  feq_dev_d2q8(mn.phip_dev, mn.ux, mn.uy, cn.inv_phi, P.rho0, en);
#pragma unroll
  for (int i = 0; i < 8; ++i) d[i] = eb[i] + dn[i] - en[i];
}

template <int PREC, bool HET>
__device__ __forceinline__ void wall_node(const StepParams& P, const typename Store<PREC>::T* src, int x, int y, int xn, int yn,
                                          int w, float ay_nb, float d[8], float& ux_nb, float& uy_nb) {
  float dn[8];
  pull_cell<PREC>(P, src, xn, yn, dn);
  wall_node_from<HET>(P, dn, x, y, xn, yn, w, ay_nb, d, ux_nb, uy_nb);
}

// Pre-collision state of any cell: the pull of Eq. 15 with its wall rules, or the extrapolated
// state of a wall node or pressure column.
template <int PREC, bool HET>
__device__ __forceinline__ void gather_cell(const StepParams& P, const typename Store<PREC>::T* src, int x, int y, float d[8]) {
  int xn, yn, w;
  float uxn, uyn;
  if (nee_node(P, x, y, xn, yn, w))
    wall_node<PREC, HET>(P, src, x, y, xn, yn, w, P.ay, d, uxn, uyn);
  else if (P.bc_x == BC_PRESSURE && (x == 0 || x == P.nx - 1))
    pressure_column<PREC, HET>(P, src, x, y, d);
  else
    pull_cell<PREC>(P, src, x, y, d);
}

// thermal equilibrium (Eq. B.6) deviation from T0/5
__device__ __forceinline__ void geq_dev(const StepParams& P, float T, float ux, float uy, float out[5]) {
  const float a = 0.2f * T - 0.2f * P.T0;
  const float b = 0.05f * P.varpi * T;
  const float hx = 0.5f * ux * T * P.inv_sigma, hy = 0.5f * uy * T * P.inv_sigma;
  out[0] = a - 4.0f * b;
  out[1] = a + hx + b;
  out[2] = a + hy + b;
  out[3] = a - hx + b;
  out[4] = a - hy + b;
}

// Pre-collision temperature of a cell: on a wall node of an extrapolated side the wall temperature
// (isothermal wall) or that of its inner neighbour (adiabatic wall), which is what the node's
// extrapolated populations sum to.
template <int PREC>
__device__ __forceinline__ double temperature_at(const StepParams& P, const typename Store<PREC>::T* gsrc, int x, int y) {
  int xn = x, yn = y, w = 0;
  if (nee_node(P, x, y, xn, yn, w) && P.Tdir[w]) return (double)P.Tw[w];
  float g[5];
  pull_cell_g<PREC>(P, gsrc, xn, yn, g);
  return (double)P.T0 + ((double)g[0] + g[1] + g[2] + g[3] + g[4]);
}

// Flow and temperature state of a wall node of a thermal context from the pulled states dn, gn of
// its nb (see gather_cell_thermal).
template <bool HET>
__device__ __forceinline__ void thermal_wall_node_from(const StepParams& P, const float dn[8], const float gn[5], int x, int y, int xn,
                                                       int yn, int w, float d[8], float g[5]) {
  const float Tn = gn[0] + gn[1] + gn[2] + gn[3] + gn[4];  // T_nb - T0
  float uxn, uyn;
  wall_node_from<HET>(P, dn, x, y, xn, yn, w, P.ay + P.g_beta * Tn, d, uxn, uyn);
  const float Tb = P.Tdir[w] ? P.Tw[w] - P.T0 : Tn;
  float eb[5], en[5];
  geq_dev(P, P.T0 + Tb, __ldg(P.uw + 2 * w), __ldg(P.uw + 2 * w + 1), eb);
  geq_dev(P, P.T0 + Tn, uxn, uyn, en);
#pragma unroll
  for (int i = 0; i < 5; ++i) g[i] = eb[i] + gn[i] - en[i];
}

// Pre-collision flow (d) and temperature (g, deviations from T0/5) state of a cell of a thermal
// context.  On a wall node of an extrapolated side, g = g_eq(T_b, u_w) + g_nb - g_eq(T_nb, u_nb)
// with T_b the wall temperature (isothermal wall) or T_nb (adiabatic wall), and the flow part
// uses the velocity of nb with the buoyancy of T_nb.
template <int PREC, bool HET>
__device__ __forceinline__ void gather_cell_thermal(const StepParams& P, const typename Store<PREC>::T* src,
                                                    const typename Store<PREC>::T* gsrc, int x, int y, float d[8], float g[5]) {
  int xn, yn, w;
  if (nee_node(P, x, y, xn, yn, w)) {
    float dn[8], gn[5];
    pull_cell<PREC>(P, src, xn, yn, dn);
    pull_cell_g<PREC>(P, gsrc, xn, yn, gn);
    thermal_wall_node_from<HET>(P, dn, gn, x, y, xn, yn, w, d, g);
  } else {
    gather_cell<PREC, HET>(P, src, x, y, d);
    pull_cell_g<PREC>(P, gsrc, x, y, g);
  }
}

}  // namespace lbm
