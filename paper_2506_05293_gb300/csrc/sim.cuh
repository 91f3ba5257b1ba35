// Internal state of a simulation and the kernel launchers shared by the
// translation units of the library.  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lattice.cuh"

namespace lbm {

enum EastMode : int { EAST_ZOUHE = 0, EAST_EXTERNAL = 1 };

// Status bits latched on the device.
enum : int { DEV_NONFINITE = 1 };

// Parameters of one launch of the fused step kernel.
struct StepParams {
  const void* src;        // populations at t (post-collision), storage type S
  void* dst;              // populations at t+1
  int32_t nx, ny;
  int64_t pitch, plane;   // elements
  const uint32_t* solid_bits;
  int32_t words_per_row;
  const uint8_t* links;   // per cell: bit i-1 set for a counted link in direction i
  double omega;
  double mrt_se, mrt_seps, mrt_sq, mrt_snu;
  double u_in, v_amp, rho_out;
  float omega_f, mrt_f[4], u_in_f, rho_out_f;   // FP32 copies for the FP32/FP16 kernels
  uint64_t seed;
  int32_t east_mode;      // EastMode
  int32_t x_periodic;
  int32_t rows;           // rows per strip (one strip = 128 columns x rows)
  int64_t t;              // absolute step index of a direct launch
  const int64_t* t_base;  // graph launches: t = *t_base + t_offset (t_base != NULL)
  int32_t t_offset;
  int32_t reduce_prev;    // the reducer block finalises the previous step's force
  int32_t prev_blocks;    // lattice blocks of the previous launch
  double* partials;       // [2 parities][partial_stride blocks][2]
  int32_t partial_stride;
  double* ring;           // 2 doubles per step
  int64_t ring_cap;
  int* status;
};

// Direct-reconstruction network on the device (FP32 and FP64 copies).
struct DevMlp {
  int n_layers = 0;
  int sizes[LBM_MLP_MAX_LAYERS + 1] = {0};
  int act = 0;
  int64_t n_params = 0;
  float* params_f = nullptr;   // W, b per layer, then in_mean[81], in_std[81]
  double* params_d = nullptr;
  float out_scale = 1.f;
};

struct NnParams {
  const void* src;
  void* dst;
  int32_t nx, ny;
  int64_t pitch, plane;
  const uint32_t* solid_bits;
  int32_t words_per_row;
  const void* net;        // float* or double* blob: layers, in_mean, in_std
  int32_t n_layers;
  int32_t sizes[LBM_MLP_MAX_LAYERS + 1];
  int32_t act;
  double out_scale;
  double rho_out, fallback_drho;
  double omega;
  double mrt_se, mrt_seps, mrt_sq, mrt_snu;
  int32_t collision;
  unsigned long long* fallbacks;
  int* status;
};

// launches blocks + 1 blocks: the last one finalises the previous step's force
void launch_step(int prec, int coll, const StepParams& p, int variant, int blocks,
                 cudaStream_t s);
// force of step tt from its block partials (prev_blocks of them) into the ring
void launch_finalize_force(const StepParams& p, int64_t tt, int blocks, cudaStream_t s);
void launch_set_t(int64_t* t_base, int64_t value, cudaStream_t s);
int step_blocks(int nx, int ny, int rows, int max_blocks);
int step_variants();
// resident blocks per GPU (occupancy x SMs) of a register-budget variant
int step_max_blocks(int prec, int coll, int variant);
void launch_geometry_prep(const uint8_t* kind, int nx, int ny, int x_periodic, uint32_t* bits,
                          int words_per_row, uint8_t* links, cudaStream_t s);
void launch_init_equilibrium(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                             const double* rho, const double* ux, const double* uy,
                             cudaStream_t s);
void launch_export(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                   double* f_out, double* rho, double* ux, double* uy, cudaStream_t s);
void launch_import(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                   const double* f_in, cudaStream_t s);
void launch_mass(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                 double* partials, int n_partials, double* out, cudaStream_t s);
void launch_nn_outflow(int prec, const NnParams& p, cudaStream_t s);

// message returned by lbm_last_error() on this thread
void set_last_error(const std::string& msg);

}  // namespace lbm

// The opaque simulation object behind the C ABI.
struct lbm_sim {
  lbm_config cfg{};
  int nx = 0, ny = 0;
  int64_t pitch = 0, plane = 0;
  size_t elem = 0;
  int prec = LBM_FP32;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;
  uint8_t* kind = nullptr;
  uint32_t* solid_bits = nullptr;
  int words_per_row = 0;
  uint8_t* links = nullptr;
  double* partials = nullptr;
  int64_t n_partials = 0;
  int partial_stride = 0;
  int64_t* t_base = nullptr;   // step index at the start of a graph chunk
  double* ring = nullptr;
  int64_t ring_cap = 0;
  int* status = nullptr;
  double* scratch_fields = nullptr;  // 9 * ny * nx doubles (import/export)
  double* mass_out = nullptr;
  unsigned long long* nn_fallbacks = nullptr;
  int64_t t_host = 0;
  int64_t drained = 0;
  bool pending = false;        // forces of step t_host - 1 not yet in the ring
  int last_blocks = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  lbm_allocator alloc{};
  bool have_alloc = false;
  int east = lbm::EAST_ZOUHE;
  int outflow = LBM_OUTFLOW_ZOUHE;
  double rho_out = 1.0;
  lbm::DevMlp nn;
  double nn_drho = 0.05;
  int rows = 8;
  int variant = 1;
  int max_blocks_v[8] = {0};
  // CUDA graphs of chunks of steps, keyed by chunk length and parity
  std::map<int64_t, cudaGraphExec_t> graphs;
  std::vector<void*> owned;   // every device allocation, freed by lbm_destroy
};
