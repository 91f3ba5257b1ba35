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
enum : int { DEV_NONFINITE = 1, DEV_TIMEOUT = 2 };

// One member lattice of a step launch (a simulation, alone or in a batch).
// Built on the host and kept in device memory; the kernels read it per block.
struct Member {
  void* buf[2];           // population buffers (storage type S); source = buf[q]
  const void* tmap[2];    // FP16 storage: tensor maps of buf[0] and buf[1] (x, y, population;
                          // 64-byte aligned, in device memory) for the row-window copies
  int32_t nx, ny, pitch, plane;   // elements; 9 * plane < 2^31
  const uint32_t* solid_bits;
  int32_t words_per_row;
  const uint8_t* links;   // per node: bit i-1 set for a counted link in direction i (a solid
                          // node: to the fluid node s - c_i; a fluid node: to the solid x + c_i)
  const uint32_t* near_bits;   // fluid nodes with a counted link (layout of solid_bits)
  double omega, mrt[6], u_in, v_amp, rho_out;   // mrt: rates of e, eps, qx, qy, pxx, pxy
  float omega_f, mrt_f[6], u_in_f, rho_out_f;   // FP32 copies for the FP32/FP16 kernels
  uint64_t seed;
  int64_t ramp_steps;     // > 0: inlet velocity u_in min(1, (t+1)/ramp_steps)
  int32_t east_mode;      // EastMode
  int32_t x_periodic;
  int32_t coll;           // lbm_collision
  int32_t tiles_x;        // 128-column tiles
  int32_t strip_first;    // first block (strip) of this member in the launch
  int32_t strip_count;    // strips of this member
  int32_t part_first;     // force partials of this member: [part_first, +part_count)
  int32_t part_count;
  int32_t blk_first;      // staged kernel: blocks of this member [blk_first, +blk_count),
  int32_t blk_count;      // strips lb, lb + blk_count, ... for local block lb
  double* ring;           // 2 doubles per step
  int64_t ring_cap;
  int* status;
  // east column rebuilt by boundary blocks (east_mode EAST_EXTERNAL):
  // ext_kind 1 = NN direct reconstruction, 2 = characteristic outflow (CBC)
  int32_t ext_kind;
  int32_t cbc_exact;      // CBC: f_0 correction that makes the density exact
  double cbc_sigma;       // CBC: sigma of Eq. 27 (sigma_max with a tuner)
  double cbc_kappa2;      // CBC: kappa2 of Eq. 26 (kappa2_max with a 2-output tuner)
  double cbc_kfac;        // CBC: (1 - M^2) c_s / length, so kappa1 = sigma * cbc_kfac
  // network of the NN outflow, or the CBC tuner (nn_layers 0: none)
  const void* nn_net;     // compute-precision blob: per layer W^T then b, in_mean, in_std
  const void* nn_bf16;    // CBC tuner: per layer W padded to [N_pad][K_pad] in BF16 (tensor cores)
  unsigned long long* nn_fallbacks;
  double nn_out_scale;
  double nn_drho;
  int32_t nn_layers;
  int32_t nn_act;
  int32_t nn_sizes[LBM_MLP_MAX_LAYERS + 1];
  int32_t nn_first;       // first boundary block of this member in the launch
  int32_t ext_rows;       // east nodes (rows) of one boundary block
  int32_t nn_blob_elems;  // floats of the network blob (copied whole into shared memory)
};

// Parameters of one launch of a step kernel.
struct StepParams {
  const Member* members;
  int32_t n_members;
  const int32_t* strip_member;   // member of each block (multi-member launches)
  int32_t rows;                  // rows per strip (one strip = 128 columns x rows)
  int32_t q;                     // index of the source buffer (members in lockstep)
  int32_t persistent;            // one member whose strips the blocks stride over
  int64_t t;                     // step index of a direct launch
  const int64_t* t_base;         // graph launches: t = *t_base + t_offset
  int32_t t_offset;
  int32_t reduce_prev;           // extra blocks finalise the previous step's forces
  double* partials;              // [2 parities][partial_stride][2]
  int32_t partial_stride;
  const int32_t* strip_force;     // per strip its force-partial slot (-1: no counted solid),
                                 // or null: one partial per block
  const int32_t* strip_order;     // one block (or claim) per strip: the strip it takes, holding
                                 // solids first; null: the natural order
  unsigned long long* dyn_ctr;   // variant 5: [next strip, finished blocks], zero between launches
  int32_t dyn_strips;            // variant 5: strips of the whole table
  int32_t nn_blocks;             // boundary blocks of the grid
  int32_t nn_blob_max;           // largest network blob (floats) of the launch's NN members
  int32_t has_cbc;               // the launch has characteristic-outflow members
  const int32_t* launch_order;   // with boundary blocks: the role of each block after the
                                 // force-reduction blocks (>= 0 stream-and-collide block,
                                 // < 0 boundary block -v - 1); null: all stream-and-collide
  const int32_t* nn_block_member;  // member of each boundary block (multi-member)
  int64_t* strip_done;           // variant 6: per strip of the table, the number of steps it
                                 // has completed; null: wait for the whole previous launch
  int64_t* reduced;              // variant 6: per member, the number of steps whose forces
                                 // are in its ring (partials of older steps may be reused)
  int32_t ext_flags;             // variant 6: strip_done index of boundary block 0's flag
  Member m0;                     // copy of the only member when n_members == 1: the
                                 // kernels then read it from the parameter bank
};

// Tensor-core network blocks of the NN outflow (FP32 and FP16 storage): a
// block takes kNnTcNodes consecutive east nodes (the rows of one mma tile)
// and stages the window of columns L-4 .. L at rows y0-2 .. y0+kNnTcNodes+1.
constexpr int kNnTcNodes = 16;
constexpr int kNnTcWin = kNnTcNodes + 4;
constexpr int kNnTcFeat = 88;        // the 81 inputs padded to a multiple of 8
constexpr int kNnTcLdIn = 92;        // row stride of the input tile (88 used; 92 = 28 mod 32
                                     // keeps the fragment loads conflict-free)
constexpr int kNnTcLdAct = 68;       // row stride of hidden activations (64 used)

// Their network blob (floats, copied whole into shared memory):
// [0, 4 kNnTcFeat): per input k < 88 the z-score shift (in_mean - w_i), the
//   inverse standard deviation, and the window offsets of its pull when the
//   node it is taken at is fluid and when it is solid (bounce-back reverses
//   the direction), as small integers; zeros for k >= 81;
// then per layer: the weights split into TF32 high and low parts in mma
//   fragment order -- for each 8-column n-tile and 8-row k-step, lane
//   (g, t) = (lane / 4, lane % 4) holds {hi W[n][k], hi W[n][k+4], lo W[n][k],
//   lo W[n][k+4]} with n = 8 ntile + g, k = 8 kstep + t (zero outside the
//   network) -- then the bias padded to a multiple of 8.
__host__ __device__ constexpr int nn_tc_pad8(int n) { return (n + 7) / 8 * 8; }
__host__ __device__ constexpr int nn_tc_layer_floats(int ni, int no) {
  return nn_tc_pad8(no) * nn_tc_pad8(ni) * 2 + nn_tc_pad8(no);
}

// Direct-reconstruction network on the device (FP32 and FP64 copies).
struct DevMlp {
  int n_layers = 0;
  int sizes[LBM_MLP_MAX_LAYERS + 1] = {0};
  int act = 0;
  int64_t n_params = 0;
  int32_t blob_elems = 0;      // per layer W^T then b, then in_mean[81], in_std[81], padded
  float* params_f = nullptr;
  double* params_d = nullptr;
  uint16_t* params_bf16 = nullptr;   // tuner only: padded BF16 weights of the tensor-core path
  int64_t bf16_elems = 0;
  float* params_tc = nullptr;        // NN outflow only: the blob of the tensor-core blocks
  int32_t tc_elems = 0;
  float out_scale = 1.f;
};


// launches blocks + n_members blocks: the extra ones finalise the previous
// step's forces; coll 0 BGK, 1 MRT, 2 per member
void launch_step(int prec, int coll, const StepParams& p, int variant, int blocks,
                 cudaStream_t s);
// forces of step tt from the block partials into each member's ring
void launch_finalize_force(const StepParams& p, int64_t tt, cudaStream_t s);
void launch_set_t(int64_t* t_base, int64_t value, cudaStream_t s);
void launch_step_ext(int prec, int coll, const StepParams& p, int variant, int blocks,
                     cudaStream_t s);   // launches with boundary blocks (step_ext.cu)
int step_strips(int nx, int ny, int rows);
int step_ext_blocks(int ny, int variant, int ext_kind, int prec);  // boundary blocks of a member
int step_ext_rows(int variant, int ext_kind, int prec);             // east nodes of one of them
bool step_variant_is_bulk(int variant);
bool step_variant_streams(int variant);   // staged variant with a fixed share per block
bool step_variant_dynamic(int variant);   // staged variant taking strips from a counter
bool step_variant_dataflow(int variant);  // staged variant ordered by per-strip completion
// every strip of the table has completed steps < t; the forces of steps < r are reduced
void launch_dataflow_reset(int64_t* strip_done, int n_strips, int64_t t, int64_t* reduced,
                           int n_members, int64_t r, cudaStream_t s);
int step_variants();
// resident blocks per GPU (occupancy x SMs) of a variant; coll 2 = per member
int step_max_blocks(int prec, int coll, int variant);
void launch_geometry_prep(const uint8_t* kind, int nx, int ny, int x_periodic, uint32_t* bits,
                          int words_per_row, uint8_t* links, uint32_t* near_bits, cudaStream_t s);

// Where f_i(x, y) of the current state lives.  mode 0: two-buffer layout,
// slot i of (x, y); 1: in-place layout after an even number of steps, slot
// opp(i) of (x, y); 2: in-place layout after an odd number, slot i of
// (x + c_ix, y + c_iy), y periodic, x periodic or into the ghost columns.
struct PopMap {
  int32_t mode = 0;
  int32_t x_periodic = 0;
};
__host__ __device__ __forceinline__ int64_t pop_offset(const PopMap& pm, int i, int x, int y,
                                                      int nx, int ny, int64_t pitch,
                                                      int64_t plane) {
  if (pm.mode == 1) return (int64_t)opp(i) * plane + (int64_t)y * pitch + x;
  if (pm.mode == 2) {
    int xs = x + cx(i), ys = y + cy(i);
    ys = ys < 0 ? ys + ny : (ys >= ny ? ys - ny : ys);
    if (pm.x_periodic) xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
    return (int64_t)i * plane + (int64_t)ys * pitch + xs;
  }
  return (int64_t)i * plane + (int64_t)y * pitch + x;
}

// rows [y0, y0 + rows) of the lattice (rows < 0: to the last row); the dense
// field and population arrays hold those rows only
void launch_init_equilibrium(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                             const double* rho, const double* ux, const double* uy,
                             cudaStream_t s, PopMap pm = PopMap{}, int y0 = 0, int rows = -1);
void launch_export(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                   double* f_out, double* rho, double* ux, double* uy, cudaStream_t s,
                   PopMap pm = PopMap{}, int y0 = 0, int rows = -1);
void launch_import(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                   const double* f_in, cudaStream_t s, PopMap pm = PopMap{}, int y0 = 0,
                   int rows = -1);
void launch_mass(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                 double* partials, int n_partials, double* out, cudaStream_t s,
                 PopMap pm = PopMap{});

// ---- in-place (AA) step (aa.cu) ----
// launches blocks + n_members (= 1) blocks like launch_step's register kernel
// variants 0-2 choose 6, 8 or 10 resident blocks per SM
void launch_aa(int prec, int coll, const StepParams& p, int variant, int blocks, cudaStream_t s);
int aa_max_blocks(int prec, int coll, int variant);

// ---- training rows and training (train.cu) ----
constexpr int kRowFloats = 84;   // 81 inputs of Eq. 15 + f_3, f_6, f_7 at the plane

struct CaptureParams {
  const void* src;                 // post-collision populations at t (pull source)
  const uint32_t* solid_bits;
  int32_t words_per_row;
  int32_t nx, ny;
  int64_t pitch, plane;
  int32_t x_t;
  float* out;                      // ny rows of kRowFloats
};
void launch_capture(int prec, const CaptureParams& p, cudaStream_t s);
void launch_snapshot(int prec, const CaptureParams& p, int n_cols, cudaStream_t s);

void dataset_stats(const float* rows, int64_t n, double* scratch, cudaStream_t s);
int dataset_stats_scratch_doubles();

struct TrainParams {
  const float* rows;               // device [n_rows][kRowFloats]
  const int32_t* order;            // device [n_steps] batch indices
  int64_t n_steps;
  int32_t batch_rows;
  int32_t n_layers;
  int32_t sizes[LBM_MLP_MAX_LAYERS + 1];
  int32_t act;
  const float* in_mean;            // device [81]
  const float* in_std;             // device [81]
  float out_scale;
  float* params;                   // device [n_params], updated in place (mode 0)
  float* adam_m;                   // device [n_params] (mode 0)
  float* adam_v;
  int64_t adam_t0;                 // Adam steps taken before this call
  float lr, beta1, beta2, eps;
  int32_t mode;                    // 0 Adam steps, 1 gradients, 2 losses only
  float* grad_out;                 // device [n_steps][n_params] (mode 1)
  double* loss_log;                // device [n_steps]
  int32_t chunk;                   // samples per shared-memory chunk (multiple of 16)
};
int train_smem_bytes(const int* sizes, int n_layers, int chunk);
int train_max_chunk(const int* sizes, int n_layers, int batch_per_cta, int smem_limit);
int train_cluster_size(const TrainParams& p, int max_cluster);
cudaError_t launch_train(const TrainParams& p, int cluster, cudaStream_t s);

// message returned by lbm_last_error() on this thread
void set_last_error(const std::string& msg);

// The six relaxed MRT rates (e, eps, qx, qy, pxx, pxy) of a config: all nine
// entries zero gives e, eps, q rates 1 and stress rates 1/tau; otherwise
// entries 1, 2, 4, 6 are taken as given and the stress rates 7, 8 default to
// 1/tau where they are zero.
inline bool mrt_rates_valid(const lbm_config& c) {
  for (int k = 0; k < 9; ++k)
    if (!(c.mrt_rates[k] >= 0.0 && c.mrt_rates[k] < 2.0)) return false;   // NaN fails too
  return true;
}
inline void mrt_rates_of(const lbm_config& c, double out[6]) {
  const double* r = c.mrt_rates;
  bool any = false;
  for (int k = 0; k < 9; ++k) any |= r[k] != 0.0;
  const double snu = 1.0 / c.tau;
  if (!any) {
    out[0] = out[1] = out[2] = out[3] = 1.0;
    out[4] = out[5] = snu;
    return;
  }
  out[0] = r[1];
  out[1] = r[2];
  out[2] = r[4];
  out[3] = r[6];
  out[4] = r[7] != 0.0 ? r[7] : snu;
  out[5] = r[8] != 0.0 ? r[8] : snu;
}

}  // namespace lbm

struct lbm_sim;

namespace lbm {

// Sims advanced together by one step launch per time step: a single sim, or
// a batch of sims of any sizes and parameters (same precision, same stream,
// in lockstep).
struct Group {
  std::vector<lbm_sim*> sims;
  bool single = true;            // the group of one lbm_sim (persistent variants allowed)
  int prec = LBM_FP32;
  int coll_mode = 0;             // 0 BGK, 1 MRT, 2 per member
  int rows = 8, variant = 1;
  cudaStream_t stream = nullptr;
  Member* d_members = nullptr;   // device launch table
  Member h_member0{};            // host copy of member 0 (single-member launches)
  int32_t* d_strip_member = nullptr;
  int32_t* d_nn_block_member = nullptr;   // member of each network block
  int nn_cap = 0;                // entries of d_nn_block_member
  unsigned long long* dyn_ctr = nullptr;   // counters of the dynamic staged variant
  int32_t* d_strip_force = nullptr;        // force-partial slot of each strip
  int32_t* d_strip_order = nullptr;        // launch order of the strips
  int32_t* d_launch_order = nullptr;       // roles of the blocks with boundary blocks
  int launch_cap = 0;                      // entries of d_launch_order
  int force_cap = 0;
  bool use_strip_force = false;
  int nn_blocks = 0;             // network blocks of the current table
  double* partials = nullptr;    // [2][partial_stride][2]
  int partial_stride = 0;
  int64_t* t_base = nullptr;
  int blocks = 0;                // lattice blocks of the current table
  bool persistent = false;
  bool aa = false;               // the in-place layout (a single member)
  int aa_max_blocks[3] = {0, 0, 0};   // resident blocks of the in-place kernel per variant
  std::vector<uint64_t> built_versions;   // member versions the table was built from
  bool pending = false;          // forces of the last launched step not yet in the rings
  // variant 6 (dataflow between consecutive step launches)
  int64_t* d_strip_done = nullptr;   // per strip: steps completed
  int64_t* d_reduced = nullptr;      // per member: steps whose forces are reduced
  int done_cap = 0;                  // strip flags (d_strip_done holds 2 done_cap entries:
                                     // strips, then boundary blocks)
  bool flow = false;                 // the current table runs the dataflow variant
  bool capturing = false;            // steps enqueued into a caller's stream capture
  int64_t flow_t = -1;               // the flags hold "steps < flow_t completed" (-1: unknown)
  int max_blocks_v[8] = {0};
  std::map<int64_t, cudaGraphExec_t> graphs;   // chunk graphs keyed by length and parity
  std::vector<void*> owned;      // allocations owned by a batch group
};

}  // namespace lbm

// The opaque simulation object behind the C ABI.
struct lbm_sim {
  lbm_config cfg{};
  int nx = 0, ny = 0;
  int64_t pitch = 0, plane = 0;
  size_t elem = 0;
  int prec = LBM_FP32;
  void* buf[2] = {nullptr, nullptr};
  const void* tmap[2] = {nullptr, nullptr};   // device tensor maps of buf[0], buf[1] (two-buffer
                                              // layout, FP16 storage)
  int cur = 0;
  uint8_t* kind = nullptr;
  uint32_t* solid_bits = nullptr;
  int words_per_row = 0;
  uint8_t* links = nullptr;
  uint32_t* near_bits = nullptr;
  int layout = LBM_LAYOUT_AB;
  void* buf_alloc = nullptr;         // AA: the allocation (buf[0] = it + one element)
  std::vector<uint8_t> solid_tile_rows;   // per 128-column tile and row: holds a counted solid
  double* ring = nullptr;
  int64_t ring_cap = 0;
  bool ring_auto = false;            // force_capacity 0: the ring grows on demand
  int* status = nullptr;
  double* scratch_fields = nullptr;  // import/export rows, allocated at first use:
  int64_t scratch_doubles = 0;       // min(9 nx ny, about 8 Mi) doubles
  double* scratch_sums = nullptr;    // ny doubles (mass rows) + 1 (total)
  unsigned long long* nn_fallbacks = nullptr;
  int64_t t_host = 0;
  int64_t drained = 0;
  uint64_t version = 1;              // bumped by every change that the launch table holds
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  lbm_allocator alloc{};
  bool have_alloc = false;
  int east = lbm::EAST_ZOUHE;
  int outflow = LBM_OUTFLOW_ZOUHE;
  double rho_out = 1.0;
  lbm::DevMlp nn;                    // NN outflow network, or the CBC tuner
  double nn_drho = 0.05;
  double cbc_sigma = 0.0, cbc_kappa2 = 0.0, cbc_mach = 0.0, cbc_length = 0.0;
  int cbc_exact = 0;
  // training-row capture (lbm_capture_plane)
  float* cap_out = nullptr;          // caller's device buffer of cap_capacity rows
  int64_t cap_capacity = 0;
  int64_t cap_rows = 0;              // rows written so far
  int32_t cap_x = 0, cap_every = 0;  // cap_every 0: not capturing
  lbm::Group own;                    // this sim alone
  lbm::Group* last_group = nullptr;  // the group that launched its last step
  int batch_refs = 0;                // batches holding this sim
  std::vector<void*> owned;          // every device allocation, freed by lbm_destroy
};

// The opaque batch object behind the C ABI.
struct lbm_batch {
  lbm::Group g;
};

namespace lbm {
// group.cu
void* dev_alloc_raw(const lbm_allocator* a, size_t bytes);
void dev_free_raw(const lbm_allocator* a, void* p);
// the process-wide default allocator (lbm_set_default_allocator); false: none
bool default_allocator(lbm_allocator* out);
void set_default_allocator(const lbm_allocator* a);
// grow an automatic force ring so that n more steps overwrite no undrained force
void sim_reserve_ring(lbm_sim* s, int64_t n);
void group_init(Group& g, const std::vector<lbm_sim*>& sims, bool single);
void group_release(Group& g);
void group_clear_graphs(Group& g);
void group_finalize(Group& g);        // enqueue the pending force reduction
void group_step(Group& g, int64_t n); // enqueue n time steps of every member
void group_set_tiling(Group& g, int rows, int variant);
float group_autotune(Group& g, int steps, int64_t flush_bytes);
void sim_settle(lbm_sim* s);          // finalise the forces of the sim's last group
struct CudaError {
  cudaError_t e;
  const char* what;
};
inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaError{e, what};
}
// the allocation holding the current state (9 plane + 256 elements): the in-place
// layout's buffer starts one element (the first ghost) before buf[0]
inline void* state_alloc(lbm_sim* s) {
  return s->layout == LBM_LAYOUT_AA ? s->buf_alloc : s->buf[s->cur];
}
// where the state after t steps keeps its populations (see PopMap)
inline PopMap pop_map(const lbm_sim* s, int64_t t) {
  PopMap pm;
  if (s->layout == LBM_LAYOUT_AA) {
    pm.mode = t % 2 == 0 ? 1 : 2;
    pm.x_periodic = s->cfg.x_periodic;
  }
  return pm;
}
}  // namespace lbm
