// Host-side declarations shared by the C-ABI layer (api.cu) and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

constexpr int kResidualMaxBlocks = 2048;  // partial-sum slots of the residual reduction

int record_error(int code, const char* msg);
}  // namespace lbm
struct lbm_config;
namespace lbm {
int validate_config(const ::lbm_config* c);
void params_from_config(const ::lbm_config& k, int prec, int pitch, int64_t plane, StepParams& P);
// The fields that differ between the lattices of a batch whose lattices share rho0, s_e, s_q and
// the storage scale (the batched per-item step then takes everything else from one lattice's
// parameters passed by value, in the kernel's constant bank, instead of staging the whole set).
struct BatchRec {
  const void* src;
  void* dst;
  const float* phi;
  const float* K;
  const float* uw;
  int64_t plane;
  int nx, ny, pitch, bc_x, bc_y, forch;
  float nu, s_v, ax, ay;
};

int64_t batch_items(int nx, int ny, int bc_y, int nt, int flat);
cudaError_t launch_step_batch_shared(const StepParams& U, const BatchRec* R, const StepParams* Pd, const int64_t* item_start,
                                     const int* item_lattice, int64_t total, int prec, int nt, int flat, cudaStream_t s);
int batch_max_ctas_per_sm(int prec, int nt);
cudaError_t launch_step_batch(const StepParams* Pd, const int64_t* item_start, const int* item_lattice, int n, int64_t total, int prec,
                              int nt, int grid, int flat, cudaStream_t s);
cudaError_t launch_step(const StepParams& P, int prec, bool het, bool thermal, cudaStream_t s);
cudaError_t launch_step_inplace(const StepParams& P, int prec, bool het, bool thermal, cudaStream_t s);
int64_t inplace_items(int nx, int ny, int bc_x, int bc_y);
cudaError_t launch_step_batch_inplace(const StepParams* Pd, const int64_t* item_start, const int* item_lattice, int64_t total, int prec,
                                      int parity, cudaStream_t s);
cudaError_t launch_put_inplace(const StepParams& P, int prec, bool het, const float* f, const float* g, bool flow, bool temp,
                               float p0, float ux0, float uy0, int phip_uniform, float T_init, cudaStream_t s);
cudaError_t launch_medium(const float* eps, const float* K, float phi_u, float K_u, int nx, int ny, int pitch, float* phi_out,
                          float* K_out, unsigned int* err, int log_k, cudaStream_t s);
cudaError_t launch_viscous_rate(const float* J, int nx, int ny, int pitch, float nu, float* sv, unsigned int* err, cudaStream_t s);
cudaError_t launch_init(const StepParams& P, int prec, bool het, bool thermal, float p0, float ux0, float uy0, int phip_uniform,
                        float T_init, bool flow, bool temp, cudaStream_t s);
cudaError_t launch_import(const StepParams& P, int prec, const float* f, const float* g, cudaStream_t s);
cudaError_t launch_export(const StepParams& P, int prec, bool het, bool thermal, float* f, float* g, cudaStream_t s);
cudaError_t launch_macros(const StepParams& P, int prec, bool het, bool thermal, float* p, float* ux, float* uy, float* T,
                          cudaStream_t s);
cudaError_t launch_copy_small(float* dst, const float* src, int n, cudaStream_t s);
cudaError_t launch_probe(const StepParams& P, int prec, bool het, bool thermal, int x, int y, float* out, cudaStream_t s);
int residual_blocks(int nx, int ny);
cudaError_t launch_residual(const StepParams& P, int prec, bool het, bool thermal, const void* prev, const void* gprev,
                            const float* uprev, double* partial, int nblocks, double* out, cudaStream_t s);
cudaError_t launch_nusselt(const StepParams& P, int prec, int side, double* out, cudaStream_t s);

cudaError_t launch_adj_seed(const StepParams& P, int prec, bool het, float* nu_out, float* g_l, float* g_phi, int kind,
                            const float* tux, const float* tuy, double* partial, int nblocks, double* loss_out, cudaStream_t s);
cudaError_t launch_adj_wall(const StepParams& P, int prec, bool het, const void* buf, float* nu, float* g_l, float* g_phi,
                            cudaStream_t s);
cudaError_t launch_adj_nee(const StepParams& P, int prec, bool het, const void* buf, float* nu, float* g_l, float* g_phi,
                           cudaStream_t s);
cudaError_t launch_adj_step(const StepParams& P, int prec, bool het, const void* buf, const float* nu_in, float* nu_out, float* g_l,
                            float* g_phi, cudaStream_t s);
cudaError_t launch_adj_init(const StepParams& P, bool het, const float* nu, float* g_phi, float p0, float ux0, float uy0,
                            int phip_uniform, cudaStream_t s);
cudaError_t launch_adj_fold(float* l32, float* p32, double* l64, double* p64, int64_t n, cudaStream_t s);

}  // namespace lbm
