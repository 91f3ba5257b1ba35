// C ABI of the library (include/lbm.h): argument checking, device memory,
// streams, CUDA-graph replay of chunks of steps, and host post-processing.
// Every numerical step of the method runs in the kernels of step.cu and nn.cu.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cmath>
#include <complex>
#include <exception>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "sim.cuh"

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

struct CudaError {
  cudaError_t e;
  const char* what;
};

inline void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw CudaError{e, what};
}

lbm_status from_cuda(const CudaError& ce) {
  g_err = std::string(ce.what) + ": " + cudaGetErrorString(ce.e);
  if (ce.e == cudaErrorMemoryAllocation) return LBM_ERR_OOM;
  return LBM_ERR_CUDA;
}

#define LBM_GUARD_BEGIN try {
#define LBM_GUARD_END                                            \
  }                                                              \
  catch (const CudaError& ce) { return from_cuda(ce); }          \
  catch (const std::bad_alloc&) { return fail(LBM_ERR_OOM, "host allocation failed"); } \
  catch (const std::exception& ex) { return fail(LBM_ERR_CUDA, ex.what()); }

constexpr int64_t kGraphChunk = 32;   // steps per captured graph (even)
constexpr int64_t kDefaultRing = int64_t(1) << 20;

void* dev_alloc(lbm_sim* s, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (s->have_alloc) {
    p = s->alloc.alloc(bytes, s->alloc.ctx);
    if (!p) throw CudaError{cudaErrorMemoryAllocation, "injected allocator"};
  } else {
    ck(cudaMalloc(&p, bytes), "cudaMalloc");
  }
  s->owned.push_back(p);
  return p;
}

void release_all(lbm_sim* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void* p : s->owned) {
    if (s->have_alloc) s->alloc.free(p, s->alloc.ctx);
    else cudaFree(p);
  }
  s->owned.clear();
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  s->stream = nullptr;
}

void clear_graphs(lbm_sim* s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

void mrt_rates(const lbm_sim* s, double& se, double& seps, double& sq, double& snu) {
  const double* r = s->cfg.mrt_rates;
  bool any = false;
  for (int k = 0; k < 9; ++k) any |= r[k] != 0.0;
  if (!any) {
    se = seps = sq = 1.0;
    snu = 1.0 / s->cfg.tau;
    return;
  }
  se = r[1];
  seps = r[2];
  sq = r[4];
  snu = r[7] != 0.0 ? r[7] : 1.0 / s->cfg.tau;
}

lbm::StepParams step_params(lbm_sim* s, int src_idx) {
  lbm::StepParams p{};
  p.src = s->buf[src_idx];
  p.dst = s->buf[1 - src_idx];
  p.nx = s->nx;
  p.ny = s->ny;
  p.pitch = s->pitch;
  p.plane = s->plane;
  p.solid_bits = s->solid_bits;
  p.words_per_row = s->words_per_row;
  p.links = s->links;
  p.omega = 1.0 / s->cfg.tau;
  mrt_rates(s, p.mrt_se, p.mrt_seps, p.mrt_sq, p.mrt_snu);
  p.u_in = s->cfg.u_in;
  p.v_amp = s->cfg.v_pert_amp;
  p.rho_out = s->rho_out;
  p.omega_f = (float)p.omega;
  p.mrt_f[0] = (float)p.mrt_se;
  p.mrt_f[1] = (float)p.mrt_seps;
  p.mrt_f[2] = (float)p.mrt_sq;
  p.mrt_f[3] = (float)p.mrt_snu;
  p.u_in_f = (float)p.u_in;
  p.rho_out_f = (float)p.rho_out;
  p.seed = s->cfg.seed;
  p.east_mode = s->east;
  p.x_periodic = s->cfg.x_periodic;
  p.rows = s->rows;
  p.partials = s->partials;
  p.partial_stride = s->partial_stride;
  p.ring = s->ring;
  p.ring_cap = s->ring_cap;
  p.status = s->status;
  return p;
}

int step_block_count(const lbm_sim* s) {
  return lbm::step_blocks(s->nx, s->ny, s->rows, s->max_blocks_v[s->variant]);
}

// Sum the force partials of the last executed step into the ring, if that
// has not happened yet (the next step's reducer block normally does it).
void finalize_force(lbm_sim* s) {
  if (!s->pending) return;
  lbm::StepParams p = step_params(s, s->cur);
  lbm::launch_finalize_force(p, s->t_host - 1, s->last_blocks, s->stream);
  ck(cudaGetLastError(), "finalize launch");
  s->pending = false;
}

// Enqueue one time step from buf[src_idx] to buf[1 - src_idx].  graph_k < 0:
// a direct launch for step t_host; graph_k >= 0: step k of a captured chunk,
// whose step index is read from t_base on the device.
void enqueue_step(lbm_sim* s, int src_idx, int graph_k = -1) {
  lbm::StepParams p = step_params(s, src_idx);
  const int blocks = step_block_count(s);
  if (graph_k < 0) {
    p.t = s->t_host;
    p.t_base = nullptr;
    p.reduce_prev = s->pending ? 1 : 0;
    p.prev_blocks = s->last_blocks;
  } else {
    p.t = 0;
    p.t_base = s->t_base;
    p.t_offset = graph_k;
    p.reduce_prev = graph_k > 0 ? 1 : 0;
    p.prev_blocks = blocks;
  }
  lbm::launch_step(s->prec, s->cfg.collision, p, s->variant, blocks, s->stream);
  if (s->east == lbm::EAST_EXTERNAL && s->outflow == LBM_OUTFLOW_NN) {
    lbm::NnParams q{};
    q.src = p.src;
    q.dst = p.dst;
    q.nx = s->nx;
    q.ny = s->ny;
    q.pitch = s->pitch;
    q.plane = s->plane;
    q.solid_bits = s->solid_bits;
    q.words_per_row = s->words_per_row;
    q.net = s->prec == LBM_FP64 ? (const void*)s->nn.params_d : (const void*)s->nn.params_f;
    q.n_layers = s->nn.n_layers;
    for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l) q.sizes[l] = s->nn.sizes[l];
    q.act = s->nn.act;
    q.out_scale = s->nn.out_scale;
    q.rho_out = s->rho_out;
    q.fallback_drho = s->nn_drho;
    q.omega = p.omega;
    q.mrt_se = p.mrt_se;
    q.mrt_seps = p.mrt_seps;
    q.mrt_sq = p.mrt_sq;
    q.mrt_snu = p.mrt_snu;
    q.collision = s->cfg.collision;
    q.fallbacks = s->nn_fallbacks;
    q.status = s->status;
    lbm::launch_nn_outflow(s->prec, q, s->stream);
  }
  ck(cudaGetLastError(), "step launch");
}

cudaGraphExec_t chunk_graph(lbm_sim* s, int64_t len) {
  const int64_t key = len * 2 + s->cur;
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) return it->second;
  cudaGraph_t g = nullptr;
  ck(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
  int idx = s->cur;
  try {
    for (int64_t k = 0; k < len; ++k) {
      enqueue_step(s, idx, (int)k);
      idx = 1 - idx;
    }
  } catch (...) {
    cudaStreamEndCapture(s->stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  ck(cudaStreamEndCapture(s->stream, &g), "end capture");
  cudaGraphExec_t ex = nullptr;
  cudaError_t e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  ck(e, "graph instantiate");
  s->graphs[key] = ex;
  return ex;
}

lbm_status check_sim(lbm_sim* s) {
  if (!s) return fail(LBM_ERR_ARG, "sim is NULL");
  if (!s->buf[0]) return fail(LBM_ERR_STATE, "sim is not initialised");
  return LBM_OK;
}

lbm_status read_status(lbm_sim* s) {
  int st = 0;
  ck(cudaMemcpyAsync(&st, s->status, sizeof(int), cudaMemcpyDeviceToHost, s->stream),
     "status copy");
  ck(cudaStreamSynchronize(s->stream), "stream sync");
  if (st & lbm::DEV_NONFINITE)
    return fail(LBM_ERR_NONFINITE, "non-finite density on the device (the run diverged)");
  return LBM_OK;
}

// Radix-2 complex FFT, in place (n a power of two).
void fft_inplace(std::vector<std::complex<double>>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const double ang = -2.0 * M_PI / (double)len;
    for (size_t i = 0; i < n; i += len) {
      for (size_t k = 0; k < len / 2; ++k) {
        const std::complex<double> w(std::cos(ang * (double)k), std::sin(ang * (double)k));
        const std::complex<double> u = a[i + k];
        const std::complex<double> v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
    }
  }
}

}  // namespace

namespace lbm {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace lbm

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

const char* lbm_version(void) { return "gb300-lbm 0.1 (sm_103a)"; }

lbm_status lbm_config_default(lbm_config* cfg) {
  if (!cfg) return fail(LBM_ERR_ARG, "cfg is NULL");
  memset(cfg, 0, sizeof(*cfg));
  cfg->nx = 64;
  cfg->ny = 64;
  cfg->tau = 0.6;
  cfg->collision = LBM_BGK;
  cfg->precision = LBM_FP32;
  cfg->rho_out = 1.0;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, lbm_sim** out) {
  if (!cfg || !out) return fail(LBM_ERR_ARG, "cfg and out must be non-NULL");
  *out = nullptr;
  if (cfg->nx < 1 || cfg->ny < 1) return fail(LBM_ERR_ARG, "nx and ny must be >= 1");
  if (!cfg->x_periodic && cfg->nx < 3) return fail(LBM_ERR_ARG, "open x needs nx >= 3");
  if ((int64_t)cfg->nx * cfg->ny > (int64_t)1 << 31)
    return fail(LBM_ERR_ARG, "lattice larger than 2^31 nodes");
  if (cfg->ny > 65535) return fail(LBM_ERR_ARG, "ny must be <= 65535");
  if ((int64_t)9 * cfg->ny * (((int64_t)cfg->nx + 63) / 64 * 64) >= ((int64_t)1 << 31))
    return fail(LBM_ERR_ARG, "9 * ny * pitch must stay below 2^31 elements");
  if (!(cfg->tau > 0.5) || !std::isfinite(cfg->tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
  if (cfg->collision != LBM_BGK && cfg->collision != LBM_MRT)
    return fail(LBM_ERR_ARG, "unknown collision");
  if (cfg->precision < LBM_FP64 || cfg->precision > LBM_FP16DEV)
    return fail(LBM_ERR_ARG, "unknown precision");
  if (!(std::fabs(cfg->u_in) < 1.0)) return fail(LBM_ERR_ARG, "|u_in| must be < 1");
  if (!(cfg->rho_out > 0.0)) return fail(LBM_ERR_ARG, "rho_out must be > 0");
  if (cfg->force_capacity < 0) return fail(LBM_ERR_ARG, "force_capacity must be >= 0");
  if (cfg->alloc && (!cfg->alloc->alloc || !cfg->alloc->free))
    return fail(LBM_ERR_ARG, "allocator needs both alloc and free");
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(cfg->mrt_rates[k]) || cfg->mrt_rates[k] < 0.0 || cfg->mrt_rates[k] >= 2.0)
      return fail(LBM_ERR_ARG, "MRT rates must lie in [0, 2)");

  lbm_sim* s = new (std::nothrow) lbm_sim();
  if (!s) return fail(LBM_ERR_OOM, "host allocation failed");
  LBM_GUARD_BEGIN
  s->cfg = *cfg;
  s->nx = cfg->nx;
  s->ny = cfg->ny;
  s->prec = cfg->precision;
  s->elem = s->prec == LBM_FP64 ? 8 : (s->prec == LBM_FP32 ? 4 : 2);
  s->pitch = ((int64_t)s->nx + 63) / 64 * 64;
  s->plane = s->pitch * s->ny;
  s->rho_out = cfg->rho_out;
  if (cfg->alloc) {
    s->alloc = *cfg->alloc;
    s->have_alloc = true;
  }
  s->cfg.alloc = nullptr;
  if (cfg->stream) {
    s->stream = (cudaStream_t)cfg->stream;
  } else {
    ck(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    s->own_stream = true;
  }
  const size_t bytes = (size_t)9 * s->plane * s->elem;
  s->buf[0] = dev_alloc(s, bytes);
  s->buf[1] = dev_alloc(s, bytes);
  const int64_t cells = (int64_t)s->nx * s->ny;
  s->kind = (uint8_t*)dev_alloc(s, cells);
  s->words_per_row = (s->nx + 31) / 32;
  s->solid_bits = (uint32_t*)dev_alloc(s, (size_t)s->words_per_row * s->ny * 4);
  s->links = (uint8_t*)dev_alloc(s, cells);
  int most = 0;
  for (int v = 0; v < lbm::step_variants(); ++v) {
    s->max_blocks_v[v] = lbm::step_max_blocks(s->prec, s->cfg.collision, v);
    if (s->max_blocks_v[v] <= 0) throw CudaError{cudaGetLastError(), "occupancy query"};
    most = std::max(most, s->max_blocks_v[v]);
  }
  // force partials: two parities x one per resident block x (Fx, Fy); the
  // mass reduction reuses them and needs ny
  s->partial_stride = most;
  s->n_partials = std::max<int64_t>((int64_t)4 * most, s->ny);
  s->partials = (double*)dev_alloc(s, (size_t)s->n_partials * sizeof(double));
  s->t_base = (int64_t*)dev_alloc(s, sizeof(int64_t));
  s->ring_cap = cfg->force_capacity > 0 ? cfg->force_capacity : kDefaultRing;
  s->ring = (double*)dev_alloc(s, (size_t)2 * s->ring_cap * sizeof(double));
  s->status = (int*)dev_alloc(s, sizeof(int));
  s->scratch_fields = (double*)dev_alloc(s, (size_t)9 * cells * sizeof(double));
  s->mass_out = (double*)dev_alloc(s, sizeof(double));
  s->nn_fallbacks = (unsigned long long*)dev_alloc(s, sizeof(unsigned long long));
  ck(cudaMemsetAsync(s->kind, 0, cells, s->stream), "memset");
  ck(cudaMemsetAsync(s->t_base, 0, sizeof(int64_t), s->stream), "memset");
  ck(cudaMemsetAsync(s->partials, 0, (size_t)s->n_partials * sizeof(double), s->stream), "memset");
  ck(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream), "memset");
  ck(cudaMemsetAsync(s->nn_fallbacks, 0, sizeof(unsigned long long), s->stream), "memset");
  ck(cudaMemsetAsync(s->ring, 0, (size_t)2 * s->ring_cap * sizeof(double), s->stream), "memset");
  // padding columns are never read by the step, but keep them defined
  ck(cudaMemsetAsync(s->buf[0], 0, bytes, s->stream), "memset");
  ck(cudaMemsetAsync(s->buf[1], 0, bytes, s->stream), "memset");
  lbm::launch_geometry_prep(s->kind, s->nx, s->ny, s->cfg.x_periodic, s->solid_bits,
                            s->words_per_row, s->links, s->stream);
  lbm::launch_init_equilibrium(s->prec, s->buf[0], s->nx, s->ny, s->pitch, s->plane, nullptr,
                               nullptr, nullptr, s->stream);
  ck(cudaGetLastError(), "init launch");
  ck(cudaStreamSynchronize(s->stream), "create sync");
  *out = s;
  return LBM_OK;
  }
  catch (const CudaError& ce) {
    lbm_status st = from_cuda(ce);
    release_all(s);
    delete s;
    return st;
  }
  catch (...) {
    release_all(s);
    delete s;
    return fail(LBM_ERR_OOM, "allocation failed");
  }
}

lbm_status lbm_destroy(lbm_sim* s) {
  if (!s) return LBM_OK;
  release_all(s);
  delete s;
  return LBM_OK;
}

lbm_status lbm_set_geometry(lbm_sim* s, const uint8_t* kind) {
  if (lbm_status st = check_sim(s)) return st;
  if (!kind) return fail(LBM_ERR_ARG, "kind is NULL");
  const int64_t cells = (int64_t)s->nx * s->ny;
  for (int64_t c = 0; c < cells; ++c)
    if (kind[c] > LBM_CELL_WALL) return fail(LBM_ERR_ARG, "cell kind must be 0, 1 or 2");
  LBM_GUARD_BEGIN
  ck(cudaMemcpyAsync(s->kind, kind, cells, cudaMemcpyHostToDevice, s->stream), "kind copy");
  lbm::launch_geometry_prep(s->kind, s->nx, s->ny, s->cfg.x_periodic, s->solid_bits,
                            s->words_per_row, s->links, s->stream);
  ck(cudaGetLastError(), "geometry launch");
  ck(cudaStreamSynchronize(s->stream), "geometry sync");
  clear_graphs(s);
  return LBM_OK;
  LBM_GUARD_END
}

static void reset_counters(lbm_sim* s) {
  s->pending = false;
  ck(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream), "memset");
  ck(cudaMemsetAsync(s->nn_fallbacks, 0, sizeof(unsigned long long), s->stream), "memset");
  s->t_host = 0;
  s->drained = 0;
}

lbm_status lbm_init_equilibrium(lbm_sim* s, const double* rho, const double* ux, const double* uy) {
  if (lbm_status st = check_sim(s)) return st;
  const int64_t cells = (int64_t)s->nx * s->ny;
  LBM_GUARD_BEGIN
  double* d = s->scratch_fields;
  const double* dr = nullptr;
  const double* du = nullptr;
  const double* dv = nullptr;
  if (rho) {
    ck(cudaMemcpyAsync(d, rho, cells * 8, cudaMemcpyHostToDevice, s->stream), "rho copy");
    dr = d;
  }
  if (ux) {
    ck(cudaMemcpyAsync(d + cells, ux, cells * 8, cudaMemcpyHostToDevice, s->stream), "ux copy");
    du = d + cells;
  }
  if (uy) {
    ck(cudaMemcpyAsync(d + 2 * cells, uy, cells * 8, cudaMemcpyHostToDevice, s->stream), "uy copy");
    dv = d + 2 * cells;
  }
  s->cur = 0;
  lbm::launch_init_equilibrium(s->prec, s->buf[0], s->nx, s->ny, s->pitch, s->plane, dr, du, dv,
                               s->stream);
  ck(cudaGetLastError(), "init launch");
  reset_counters(s);
  ck(cudaStreamSynchronize(s->stream), "init sync");
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_set_outflow_zouhe(lbm_sim* s, double rho_out) {
  if (lbm_status st = check_sim(s)) return st;
  if (!(rho_out > 0.0) || !std::isfinite(rho_out)) return fail(LBM_ERR_ARG, "rho_out must be > 0");
  if (s->cfg.x_periodic) return fail(LBM_ERR_STATE, "x is periodic: there is no outflow");
  s->rho_out = rho_out;
  s->east = lbm::EAST_ZOUHE;
  s->outflow = LBM_OUTFLOW_ZOUHE;
  clear_graphs(s);
  return LBM_OK;
}

lbm_status lbm_set_outflow_nn(lbm_sim* s, const lbm_mlp* net, double fallback_drho) {
  if (lbm_status st = check_sim(s)) return st;
  if (!net || !net->params) return fail(LBM_ERR_ARG, "net and net->params must be non-NULL");
  if (s->cfg.x_periodic) return fail(LBM_ERR_STATE, "x is periodic: there is no outflow");
  if (s->nx < 5) return fail(LBM_ERR_ARG, "the NN outflow needs nx >= 5");
  if (net->n_layers < 1 || net->n_layers > LBM_MLP_MAX_LAYERS)
    return fail(LBM_ERR_ARG, "n_layers must be 1..4");
  if (net->sizes[0] != 81 || net->sizes[net->n_layers] != 3)
    return fail(LBM_ERR_ARG, "the direct-reconstruction net maps 81 inputs to 3 outputs");
  int64_t np = 0;
  for (int l = 0; l < net->n_layers; ++l) {
    if (net->sizes[l + 1] < 1 || (l < net->n_layers - 1 && net->sizes[l + 1] > 64))
      return fail(LBM_ERR_ARG, "hidden layers must have 1..64 units");
    np += (int64_t)net->sizes[l] * net->sizes[l + 1] + net->sizes[l + 1];
  }
  if (net->n_params != np) return fail(LBM_ERR_ARG, "n_params does not match the layer sizes");
  if (net->act != 0 && net->act != 1) return fail(LBM_ERR_ARG, "act must be 0 (tanh) or 1 (leaky)");
  if (!(fallback_drho > 0.0)) return fail(LBM_ERR_ARG, "fallback_drho must be > 0");
  if (!std::isfinite(net->out_scale)) return fail(LBM_ERR_ARG, "out_scale must be finite");
  for (int64_t k = 0; k < np; ++k)
    if (!std::isfinite(net->params[k])) return fail(LBM_ERR_ARG, "non-finite network parameter");
  std::vector<float> blob(np + 2 * 81);
  memcpy(blob.data(), net->params, np * sizeof(float));
  for (int k = 0; k < 81; ++k) {
    blob[np + k] = net->in_mean ? net->in_mean[k] : 0.f;
    const float sd = net->in_std ? net->in_std[k] : 1.f;
    if (!(sd > 0.f) || !std::isfinite(sd)) return fail(LBM_ERR_ARG, "in_std must be > 0");
    blob[np + 81 + k] = sd;
  }
  LBM_GUARD_BEGIN
  if (!s->nn.params_f || s->nn.n_params != np) {
    s->nn.params_f = (float*)dev_alloc(s, blob.size() * sizeof(float));
    s->nn.params_d = (double*)dev_alloc(s, blob.size() * sizeof(double));
  }
  std::vector<double> blob_d(blob.begin(), blob.end());
  ck(cudaMemcpyAsync(s->nn.params_f, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice,
                     s->stream), "net copy");
  ck(cudaMemcpyAsync(s->nn.params_d, blob_d.data(), blob_d.size() * 8, cudaMemcpyHostToDevice,
                     s->stream), "net copy");
  ck(cudaStreamSynchronize(s->stream), "net sync");
  s->nn.n_layers = net->n_layers;
  for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l) s->nn.sizes[l] = l <= net->n_layers ? net->sizes[l] : 0;
  s->nn.act = net->act;
  s->nn.n_params = np;
  s->nn.out_scale = net->out_scale;
  s->nn_drho = fallback_drho;
  s->east = lbm::EAST_EXTERNAL;
  s->outflow = LBM_OUTFLOW_NN;
  clear_graphs(s);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_nn_fallbacks(lbm_sim* s, int64_t* count) {
  if (lbm_status st = check_sim(s)) return st;
  if (!count) return fail(LBM_ERR_ARG, "count is NULL");
  LBM_GUARD_BEGIN
  unsigned long long c = 0;
  ck(cudaMemcpyAsync(&c, s->nn_fallbacks, sizeof(c), cudaMemcpyDeviceToHost, s->stream), "copy");
  ck(cudaStreamSynchronize(s->stream), "sync");
  *count = (int64_t)c;
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_step(lbm_sim* s, int64_t n) {
  if (lbm_status st = check_sim(s)) return st;
  if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
  LBM_GUARD_BEGIN
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  ck(cudaStreamIsCapturing(s->stream, &cap), "capture query");
  const bool use_graphs = cap == cudaStreamCaptureStatusNone;
  while (n > 0) {
    if (use_graphs && n >= kGraphChunk) {
      cudaGraphExec_t ex = chunk_graph(s, kGraphChunk);
      finalize_force(s);
      lbm::launch_set_t(s->t_base, s->t_host, s->stream);
      ck(cudaGetLastError(), "set_t launch");
      ck(cudaGraphLaunch(ex, s->stream), "graph launch");
      n -= kGraphChunk;
      s->t_host += kGraphChunk;
    } else {
      enqueue_step(s, s->cur);
      s->cur = 1 - s->cur;
      n -= 1;
      s->t_host += 1;
    }
    s->pending = true;
    s->last_blocks = step_block_count(s);
  }
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_sync(lbm_sim* s) {
  if (lbm_status st = check_sim(s)) return st;
  LBM_GUARD_BEGIN
  finalize_force(s);
  return read_status(s);
  LBM_GUARD_END
}

lbm_status lbm_time(lbm_sim* s, int64_t* t) {
  if (lbm_status st = check_sim(s)) return st;
  if (!t) return fail(LBM_ERR_ARG, "t is NULL");
  *t = s->t_host;
  return LBM_OK;
}

lbm_status lbm_forces(lbm_sim* s, double* fx, double* fy, int64_t cap, int64_t* n_out) {
  if (lbm_status st = check_sim(s)) return st;
  if (!n_out || cap < 0 || (cap > 0 && (!fx || !fy)))
    return fail(LBM_ERR_ARG, "fx, fy and n_out must be non-NULL and cap >= 0");
  LBM_GUARD_BEGIN
  *n_out = 0;
  finalize_force(s);
  lbm_status st = read_status(s);
  int64_t avail = s->t_host - s->drained;
  int64_t start = s->drained;
  if (avail > s->ring_cap) {
    start = s->t_host - s->ring_cap;
    avail = s->ring_cap;
  }
  const int64_t take = std::min(avail, cap);
  std::vector<double> tmp((size_t)2 * std::max<int64_t>(take, 1));
  int64_t done = 0;
  while (done < take) {
    const int64_t k = (start + done) % s->ring_cap;
    const int64_t seg = std::min(take - done, s->ring_cap - k);
    ck(cudaMemcpyAsync(tmp.data() + 2 * done, s->ring + 2 * k, (size_t)seg * 16,
                       cudaMemcpyDeviceToHost, s->stream), "force copy");
    done += seg;
  }
  ck(cudaStreamSynchronize(s->stream), "force sync");
  for (int64_t k = 0; k < take; ++k) {
    fx[k] = tmp[2 * k];
    fy[k] = tmp[2 * k + 1];
  }
  s->drained = start + take;
  *n_out = take;
  return st;
  LBM_GUARD_END
}

lbm_status lbm_fields(lbm_sim* s, double* rho, double* ux, double* uy) {
  if (lbm_status st = check_sim(s)) return st;
  const int64_t cells = (int64_t)s->nx * s->ny;
  LBM_GUARD_BEGIN
  double* d = s->scratch_fields;
  lbm::launch_export(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane, nullptr, d,
                     d + cells, d + 2 * cells, s->stream);
  ck(cudaGetLastError(), "export launch");
  if (rho) ck(cudaMemcpyAsync(rho, d, cells * 8, cudaMemcpyDeviceToHost, s->stream), "copy");
  if (ux) ck(cudaMemcpyAsync(ux, d + cells, cells * 8, cudaMemcpyDeviceToHost, s->stream), "copy");
  if (uy) ck(cudaMemcpyAsync(uy, d + 2 * cells, cells * 8, cudaMemcpyDeviceToHost, s->stream), "copy");
  return read_status(s);
  LBM_GUARD_END
}

lbm_status lbm_get_populations(lbm_sim* s, double* f) {
  if (lbm_status st = check_sim(s)) return st;
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  const int64_t cells = (int64_t)s->nx * s->ny;
  LBM_GUARD_BEGIN
  lbm::launch_export(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane,
                     s->scratch_fields, nullptr, nullptr, nullptr, s->stream);
  ck(cudaGetLastError(), "export launch");
  ck(cudaMemcpyAsync(f, s->scratch_fields, 9 * cells * 8, cudaMemcpyDeviceToHost, s->stream),
     "copy");
  return read_status(s);
  LBM_GUARD_END
}

lbm_status lbm_set_populations(lbm_sim* s, const double* f) {
  if (lbm_status st = check_sim(s)) return st;
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  const int64_t cells = (int64_t)s->nx * s->ny;
  LBM_GUARD_BEGIN
  ck(cudaMemcpyAsync(s->scratch_fields, f, 9 * cells * 8, cudaMemcpyHostToDevice, s->stream),
     "copy");
  lbm::launch_import(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane,
                     s->scratch_fields, s->stream);
  ck(cudaGetLastError(), "import launch");
  ck(cudaStreamSynchronize(s->stream), "sync");
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_mass(lbm_sim* s, double* mass) {
  if (lbm_status st = check_sim(s)) return st;
  if (!mass) return fail(LBM_ERR_ARG, "mass is NULL");
  LBM_GUARD_BEGIN
  lbm::launch_mass(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane, s->partials,
                   (int)s->n_partials, s->mass_out, s->stream);
  ck(cudaGetLastError(), "mass launch");
  ck(cudaMemcpyAsync(mass, s->mass_out, 8, cudaMemcpyDeviceToHost, s->stream), "copy");
  return read_status(s);
  LBM_GUARD_END
}

lbm_status lbm_device_state(lbm_sim* s, void** base, int64_t* pitch, int64_t* plane) {
  if (lbm_status st = check_sim(s)) return st;
  if (!base || !pitch || !plane) return fail(LBM_ERR_ARG, "outputs must be non-NULL");
  *base = s->buf[s->cur];
  *pitch = s->pitch;
  *plane = s->plane;
  return LBM_OK;
}

lbm_status lbm_set_tiling(lbm_sim* s, int32_t rows, int32_t variant) {
  if (lbm_status st = check_sim(s)) return st;
  if (rows < 1 || rows > 64) return fail(LBM_ERR_ARG, "rows must be in 1..64");
  if (variant < 0 || variant >= lbm::step_variants()) return fail(LBM_ERR_ARG, "bad variant");
  LBM_GUARD_BEGIN
  finalize_force(s);
  LBM_GUARD_END
  s->rows = rows;
  s->variant = variant;
  clear_graphs(s);
  return LBM_OK;
}

lbm_status lbm_get_tiling(lbm_sim* s, int32_t* rows, int32_t* variant) {
  if (lbm_status st = check_sim(s)) return st;
  if (!rows || !variant) return fail(LBM_ERR_ARG, "outputs must be non-NULL");
  *rows = s->rows;
  *variant = s->variant;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_sim* s, int32_t steps, int64_t flush_bytes, float* best_ms) {
  if (lbm_status st = check_sim(s)) return st;
  if (steps < 1 || steps > 10000) return fail(LBM_ERR_ARG, "steps must be in 1..10000");
  if (flush_bytes < 0) return fail(LBM_ERR_ARG, "flush_bytes must be >= 0");
  void* snap = nullptr;
  void* flush = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto cleanup = [&]() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (snap) cudaFree(snap);
    if (flush) cudaFree(flush);
  };
  try {
    const size_t bytes = (size_t)9 * s->plane * s->elem;
    ck(cudaStreamSynchronize(s->stream), "sync");
    ck(cudaMalloc(&snap, bytes), "autotune snapshot");
    if (flush_bytes > 0) ck(cudaMalloc(&flush, (size_t)flush_bytes), "autotune flush buffer");
    ck(cudaEventCreate(&e0), "event");
    ck(cudaEventCreate(&e1), "event");
    finalize_force(s);
    const int cur0 = s->cur;
    unsigned long long fb0 = 0;
    int st0 = 0;
    ck(cudaMemcpyAsync(snap, s->buf[cur0], bytes, cudaMemcpyDeviceToDevice, s->stream), "snapshot");
    ck(cudaMemcpyAsync(&fb0, s->nn_fallbacks, 8, cudaMemcpyDeviceToHost, s->stream), "snapshot");
    ck(cudaMemcpyAsync(&st0, s->status, 4, cudaMemcpyDeviceToHost, s->stream), "snapshot");
    ck(cudaStreamSynchronize(s->stream), "sync");
    const int64_t t_host0 = s->t_host, drained0 = s->drained;
    auto restore = [&]() {
      s->cur = cur0;
      ck(cudaMemcpyAsync(s->buf[cur0], snap, bytes, cudaMemcpyDeviceToDevice, s->stream), "restore");
      ck(cudaMemcpyAsync(s->nn_fallbacks, &fb0, 8, cudaMemcpyHostToDevice, s->stream), "restore");
      ck(cudaMemcpyAsync(s->status, &st0, 4, cudaMemcpyHostToDevice, s->stream), "restore");
      ck(cudaStreamSynchronize(s->stream), "sync");
      s->t_host = t_host0;
      s->drained = drained0;
      s->pending = false;
    };
    const int rows_c[] = {2, 4, 8, 16, 32};
    float best = 1e30f;
    int best_rows = s->rows, best_var = s->variant;
    for (int v = 0; v < lbm::step_variants(); ++v) {
      for (int r : rows_c) {
        s->rows = r;
        s->variant = v;
        for (int w = 0; w < 2; ++w) {
          enqueue_step(s, s->cur);
          s->cur = 1 - s->cur;
          s->t_host += 1;
          s->pending = true;
          s->last_blocks = step_block_count(s);
        }
        float total = 0.f;
        for (int k = 0; k < steps; ++k) {
          if (flush) ck(cudaMemsetAsync(flush, k & 0xff, (size_t)flush_bytes, s->stream), "flush");
          ck(cudaEventRecord(e0, s->stream), "event");
          enqueue_step(s, s->cur);
          s->cur = 1 - s->cur;
          s->t_host += 1;
          s->pending = true;
          s->last_blocks = step_block_count(s);
          ck(cudaEventRecord(e1, s->stream), "event");
          ck(cudaEventSynchronize(e1), "event sync");
          float ms = 0.f;
          ck(cudaEventElapsedTime(&ms, e0, e1), "event time");
          total += ms;
        }
        const float mean = total / (float)steps;
        if (mean < best) {
          best = mean;
          best_rows = r;
          best_var = v;
        }
        restore();
      }
    }
    s->rows = best_rows;
    s->variant = best_var;
    clear_graphs(s);
    if (best_ms) *best_ms = best;
    cleanup();
    return LBM_OK;
  } catch (const CudaError& ce) {
    cleanup();
    return from_cuda(ce);
  }
}

lbm_status lbm_strouhal(const double* cl, int64_t n, double length, double u, double* st) {
  if (!cl || !st) return fail(LBM_ERR_ARG, "cl and st must be non-NULL");
  if (n < 8) return fail(LBM_ERR_ARG, "need at least 8 samples");
  if (!(u != 0.0) || !std::isfinite(u) || !std::isfinite(length))
    return fail(LBM_ERR_ARG, "length and u must be finite, u != 0");
  try {
    int64_t m = 1;
    while (m * 2 <= n) m *= 2;
    const double* x = cl + (n - m);
    double mean = 0.0;
    for (int64_t k = 0; k < m; ++k) mean += x[k];
    mean /= (double)m;
    std::vector<std::complex<double>> a((size_t)m);
    for (int64_t k = 0; k < m; ++k) {
      const double w = 0.5 - 0.5 * std::cos(2.0 * M_PI * (double)k / (double)m);
      a[(size_t)k] = std::complex<double>((x[k] - mean) * w, 0.0);
    }
    fft_inplace(a);
    const int64_t nb = m / 2 + 1;
    std::vector<double> mag((size_t)nb);
    for (int64_t k = 0; k < nb; ++k) mag[(size_t)k] = std::abs(a[(size_t)k]);
    int64_t kp = 1;
    for (int64_t k = 2; k < nb; ++k)
      if (mag[(size_t)k] > mag[(size_t)kp]) kp = k;
    double delta = 0.0;
    if (kp - 1 >= 1 && kp + 1 < nb) {
      const double den = mag[kp - 1] - 2.0 * mag[kp] + mag[kp + 1];
      if (den != 0.0) delta = 0.5 * (mag[kp - 1] - mag[kp + 1]) / den;
    }
    const double f = ((double)kp + delta) / (double)m;
    *st = f * length / u;
    return LBM_OK;
  } catch (...) {
    return fail(LBM_ERR_OOM, "host allocation failed");
  }
}

}  // extern "C"
