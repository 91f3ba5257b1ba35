// C ABI of the library (include/lbm.h): argument checking, device memory,
// streams, CUDA-graph replay of chunks of steps, and host post-processing.
// Every numerical step of the method runs in the kernels of step.cu and train.cu.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <complex>
#include <exception>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "sim.cuh"

namespace {

using lbm::CudaError;
using lbm::ck;

thread_local std::string g_err;

lbm_status fail(lbm_status s, const std::string& msg) {
  g_err = msg;
  return s;
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

// force ring of a sim created with force_capacity 0: it starts at this many
// steps and grows on demand (see lbm::sim_reserve_ring)
constexpr int64_t kInitialRing = int64_t(1) << 12;
// import/export scratch: at most this many doubles (64 MiB), whole rows
constexpr int64_t kScratchDoubles = int64_t(8) << 20;

void* dev_alloc(lbm_sim* s, size_t bytes) {
  void* p = lbm::dev_alloc_raw(s->have_alloc ? &s->alloc : nullptr, bytes);
  s->owned.push_back(p);
  return p;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the library
// does not link the driver library itself)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// The tensor maps of the two population buffers (FP16 storage) for the staged
// kernel's row-window copies: a 3-D view (x: pitch elements, y: ny rows, population: 9 planes)
// with a box of 128 + 2 A columns, one row and nine populations, A = 16 bytes
// in elements (the kernel's row window).  Stored in 256 bytes of device
// memory, each map 64-byte aligned.
void make_tensor_maps(lbm_sim* s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) throw lbm::CudaError{cudaErrorNotSupported, "cuTensorMapEncodeTiled unavailable"};
  unsigned char* d = static_cast<unsigned char*>(dev_alloc(s, 256 + 64));
  d += (64 - (reinterpret_cast<uintptr_t>(d) & 63)) & 63;
  const CUtensorMapDataType dt = s->prec == LBM_FP64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                               : s->prec == LBM_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                     : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  const cuuint64_t dims[3] = {(cuuint64_t)s->pitch, (cuuint64_t)s->ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)s->pitch * s->elem, (cuuint64_t)s->plane * s->elem};
  const cuuint32_t box[3] = {(cuuint32_t)(128 + 2 * (16 / s->elem)), 1, 9};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap maps[2];
  for (int b = 0; b < 2; ++b) {
    const CUresult r = enc(&maps[b], dt, 3, s->buf[b], dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw lbm::CudaError{cudaErrorInvalidValue, "tensor map encoding"};
  }
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  ck(cudaMemcpyAsync(d, maps, sizeof(maps), cudaMemcpyHostToDevice, s->stream),
     "tensor map copy");
  ck(cudaStreamSynchronize(s->stream), "tensor map copy");
  s->tmap[0] = d;
  s->tmap[1] = d + 128;
}

// Scratch for row chunks of per_node doubles per node: allocated at the first
// import or export, min(9 nx ny, kScratchDoubles) doubles but at least one row
// of nine populations.  *rows gets the rows one chunk holds.
double* field_scratch(lbm_sim* s, int per_node, int* rows) {
  if (!s->scratch_fields) {
    const int64_t cells = (int64_t)s->nx * s->ny;
    const int64_t want =
        std::min<int64_t>(9 * cells, std::max<int64_t>(kScratchDoubles, 9 * (int64_t)s->nx));
    s->scratch_fields = (double*)dev_alloc(s, (size_t)want * sizeof(double));
    s->scratch_doubles = want;
  }
  *rows = (int)std::max<int64_t>(
      1, std::min<int64_t>(s->ny, s->scratch_doubles / ((int64_t)per_node * s->nx)));
  return s->scratch_fields;
}

void release_all(lbm_sim* s) {
  lbm::group_release(s->own);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void* p : s->owned) lbm::dev_free_raw(s->have_alloc ? &s->alloc : nullptr, p);
  s->owned.clear();
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  s->stream = nullptr;
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
  if (st & lbm::DEV_TIMEOUT)
    return fail(LBM_ERR_TIMEOUT,
                "a bounded device wait gave up (bulk-copy pipeline or dataflow flags)");
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

namespace {

// Device buffer freed when the scope ends (training calls own their memory),
// taken from the process-wide default allocator (lbm_set_default_allocator).
struct DevBuf {
  void* p = nullptr;
  lbm_allocator a{};
  bool have = false;
  explicit DevBuf(size_t bytes) {
    have = lbm::default_allocator(&a);
    p = lbm::dev_alloc_raw(have ? &a : nullptr, bytes ? bytes : 16);
  }
  ~DevBuf() {
    // an injected allocator may hand the memory out again at once: on an
    // early exit kernels of this call could still be using it
    if (have && p) cudaDeviceSynchronize();
    lbm::dev_free_raw(have ? &a : nullptr, p);
  }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

lbm_status check_train_net(const lbm_mlp* net, int64_t* n_params) {
  if (!net || !net->params) return fail(LBM_ERR_ARG, "net and net->params must be non-NULL");
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
  if (!std::isfinite(net->out_scale)) return fail(LBM_ERR_ARG, "out_scale must be finite");
  for (int64_t k = 0; k < np; ++k)
    if (!std::isfinite(net->params[k])) return fail(LBM_ERR_ARG, "non-finite network parameter");
  for (int k = 0; k < 81; ++k) {
    const float sd = net->in_std ? net->in_std[k] : 1.f;
    if (!(sd > 0.f) || !std::isfinite(sd)) return fail(LBM_ERR_ARG, "in_std must be > 0");
    if (net->in_mean && !std::isfinite(net->in_mean[k]))
      return fail(LBM_ERR_ARG, "in_mean must be finite");
  }
  *n_params = np;
  return LBM_OK;
}

lbm_status check_train_args(const float* rows, int64_t n_rows, const int32_t* order,
                            int64_t n_steps, const lbm_train_opts* o) {
  if (!rows || !order || !o) return fail(LBM_ERR_ARG, "rows, order and opts must be non-NULL");
  if (o->batch_rows < 1) return fail(LBM_ERR_ARG, "batch_rows must be >= 1");
  if (n_rows < o->batch_rows) return fail(LBM_ERR_ARG, "n_rows is below one batch");
  if (n_steps < 0) return fail(LBM_ERR_ARG, "n_steps must be >= 0");
  const int64_t n_batches = n_rows / o->batch_rows;
  for (int64_t k = 0; k < n_steps; ++k)
    if (order[k] < 0 || order[k] >= n_batches) return fail(LBM_ERR_ARG, "batch index out of range");
  if (!(o->lr > 0.0) || !(o->eps > 0.0) || !(o->beta1 >= 0.0 && o->beta1 < 1.0) ||
      !(o->beta2 >= 0.0 && o->beta2 < 1.0))
    return fail(LBM_ERR_ARG, "Adam needs lr > 0, eps > 0, 0 <= beta1, beta2 < 1");
  if (o->adam_t0 < 0) return fail(LBM_ERR_ARG, "adam_t0 must be >= 0");
  if (o->max_cluster < 0 || o->max_cluster > 16)
    return fail(LBM_ERR_ARG, "max_cluster must be 0..16");
  return LBM_OK;
}

constexpr int64_t kTrainStepsPerLaunch = 4096;

// Shared part of lbm_nn_train (mode 0) and lbm_nn_loss_grad (mode 1 or 2).
lbm_status run_training(const float* rows, int64_t n_rows, const int32_t* order, int64_t n_steps,
                        const lbm_train_opts* o, const lbm_mlp* net, int mode, float* params_out,
                        float* adam_m, float* adam_v, double* losses, float* grads) {
  int64_t np = 0;
  if (lbm_status st = check_train_net(net, &np)) return st;
  if (lbm_status st = check_train_args(rows, n_rows, order, n_steps, o)) return st;
  if (n_steps == 0) {
    if (params_out) memcpy(params_out, net->params, np * sizeof(float));
    return LBM_OK;
  }
  LBM_GUARD_BEGIN
  cudaStream_t stream = static_cast<cudaStream_t>(o->stream);
  int dev = 0, smem_limit = 0;
  ck(cudaGetDevice(&dev), "device");
  ck(cudaDeviceGetAttribute(&smem_limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "attr");
  lbm::TrainParams p{};
  p.batch_rows = o->batch_rows;
  p.n_layers = net->n_layers;
  for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l) p.sizes[l] = l <= net->n_layers ? net->sizes[l] : 0;
  p.act = net->act;
  p.out_scale = net->out_scale;
  p.lr = (float)o->lr;
  p.beta1 = (float)o->beta1;
  p.beta2 = (float)o->beta2;
  p.eps = (float)o->eps;
  p.mode = mode;
  p.rows = rows;
  const int max_c = o->max_cluster > 0 ? o->max_cluster : 16;
  p.chunk = lbm::train_max_chunk(p.sizes, p.n_layers, (o->batch_rows + max_c - 1) / max_c,
                                 smem_limit);
  if (p.chunk <= 0) return fail(LBM_ERR_UNSUPPORTED, "network too large for shared memory");
  int cluster = lbm::train_cluster_size(p, max_c);
  if (cluster <= 0) return fail(LBM_ERR_UNSUPPORTED, "no cluster of the training kernel fits");
  p.chunk = lbm::train_max_chunk(p.sizes, p.n_layers, (o->batch_rows + cluster - 1) / cluster,
                                 smem_limit);
  if (p.chunk <= 0) return fail(LBM_ERR_UNSUPPORTED, "network too large for shared memory");

  const int64_t per_launch = std::min<int64_t>(n_steps, kTrainStepsPerLaunch);
  DevBuf d_params(np * sizeof(float)), d_m(np * sizeof(float)), d_v(np * sizeof(float));
  DevBuf d_mean(81 * sizeof(float)), d_std(81 * sizeof(float));
  DevBuf d_order(n_steps * sizeof(int32_t)), d_loss(per_launch * sizeof(double));
  DevBuf d_grad(mode == 1 ? per_launch * np * sizeof(float) : 16);
  std::vector<float> mean(81), sd(81);
  for (int k = 0; k < 81; ++k) {
    mean[k] = net->in_mean ? net->in_mean[k] : 0.f;
    sd[k] = net->in_std ? net->in_std[k] : 1.f;
  }
  ck(cudaMemcpyAsync(d_params.p, net->params, np * 4, cudaMemcpyHostToDevice, stream), "copy");
  ck(cudaMemcpyAsync(d_mean.p, mean.data(), 81 * 4, cudaMemcpyHostToDevice, stream), "copy");
  ck(cudaMemcpyAsync(d_std.p, sd.data(), 81 * 4, cudaMemcpyHostToDevice, stream), "copy");
  ck(cudaMemcpyAsync(d_order.p, order, n_steps * 4, cudaMemcpyHostToDevice, stream), "copy");
  if (adam_m) ck(cudaMemcpyAsync(d_m.p, adam_m, np * 4, cudaMemcpyHostToDevice, stream), "copy");
  else ck(cudaMemsetAsync(d_m.p, 0, np * 4, stream), "memset");
  if (adam_v) ck(cudaMemcpyAsync(d_v.p, adam_v, np * 4, cudaMemcpyHostToDevice, stream), "copy");
  else ck(cudaMemsetAsync(d_v.p, 0, np * 4, stream), "memset");
  p.in_mean = d_mean.as<float>();
  p.in_std = d_std.as<float>();
  p.params = d_params.as<float>();
  p.adam_m = d_m.as<float>();
  p.adam_v = d_v.as<float>();
  p.grad_out = d_grad.as<float>();
  p.loss_log = d_loss.as<double>();
  for (int64_t k0 = 0; k0 < n_steps; k0 += per_launch) {
    p.n_steps = std::min(per_launch, n_steps - k0);
    p.order = d_order.as<int32_t>() + k0;
    p.adam_t0 = o->adam_t0 + k0;
    ck(lbm::launch_train(p, cluster, stream), "training launch");
    if (losses)
      ck(cudaMemcpyAsync(losses + k0, d_loss.p, p.n_steps * sizeof(double),
                         cudaMemcpyDeviceToHost, stream), "loss copy");
    if (mode == 1 && grads)
      ck(cudaMemcpyAsync(grads + k0 * np, d_grad.p, p.n_steps * np * sizeof(float),
                         cudaMemcpyDeviceToHost, stream), "grad copy");
    ck(cudaStreamSynchronize(stream), "training sync");
  }
  if (mode == 0) {
    if (params_out)
      ck(cudaMemcpy(params_out, d_params.p, np * 4, cudaMemcpyDeviceToHost), "copy");
    if (adam_m) ck(cudaMemcpy(adam_m, d_m.p, np * 4, cudaMemcpyDeviceToHost), "copy");
    if (adam_v) ck(cudaMemcpy(adam_v, d_v.p, np * 4, cudaMemcpyDeviceToHost), "copy");
  }
  return LBM_OK;
  LBM_GUARD_END
}

}  // namespace

namespace {

// Copy a network to the device as the blob the boundary blocks read: per
// layer W transposed (row k = input k's weights to every unit) then b; then
// in_mean[n_in], in_std[n_in]; padded to a multiple of 4 elements; FP32 and
// FP64 copies.  Layer sizes are checked by the caller.
// IEEE binary32 -> bfloat16, round to nearest even (finite inputs)
uint16_t bf16_rn(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

// IEEE binary32 -> TF32 (10 mantissa bits), round to nearest with ties away
// from zero, as the device's cvt.rna.tf32.f32 (finite inputs): the result is
// a binary32 value whose 13 low mantissa bits are zero
float tf32_rna_host(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  memcpy(&f, &u, 4);
  return f;
}

// The blob of the NN outflow's tensor-core blocks (layout at nn_tc_layer_floats
// in sim.cuh): input constants, then per layer the TF32-split weights in mma
// fragment order and the padded bias.
std::vector<float> nn_tc_blob(const lbm_mlp* net) {
  using namespace lbm;
  int64_t n = 4 * kNnTcFeat;
  for (int l = 0; l < net->n_layers; ++l) n += nn_tc_layer_floats(net->sizes[l], net->sizes[l + 1]);
  std::vector<float> b((size_t)n, 0.f);
  for (int kx = 0; kx < 81; ++kx) {
    const int col = kx / 27, j = (kx / 9) % 3, i = kx % 9, o = opp(i), c = 3 - col;
    const float mean = net->in_mean ? net->in_mean[kx] : 0.f;
    const float sd = net->in_std ? net->in_std[kx] : 1.f;
    b[(size_t)kx] = mean - wgt<float>(i);
    b[(size_t)(kNnTcFeat + kx)] = 1.f / sd;
    b[(size_t)(2 * kNnTcFeat + kx)] = (float)((i * kNnTcWin + j + 1 - cy(i)) * 5 + c - cx(i));
    b[(size_t)(3 * kNnTcFeat + kx)] = (float)((o * kNnTcWin + j + 1 - cy(o)) * 5 + c - cx(o));
  }
  int64_t off = 4 * kNnTcFeat, poff = 0;
  for (int l = 0; l < net->n_layers; ++l) {
    const int ni = net->sizes[l], no = net->sizes[l + 1];
    const int K8 = nn_tc_pad8(ni) / 8, N8 = nn_tc_pad8(no) / 8;
    const float* W = net->params + poff;   // [no][ni]
    for (int jt = 0; jt < N8; ++jt)
      for (int kk = 0; kk < K8; ++kk)
        for (int lane = 0; lane < 32; ++lane) {
          const int nn = jt * 8 + lane / 4, k = kk * 8 + lane % 4;
          const float w0 = nn < no && k < ni ? W[(int64_t)nn * ni + k] : 0.f;
          const float w1 = nn < no && k + 4 < ni ? W[(int64_t)nn * ni + k + 4] : 0.f;
          const float h0 = tf32_rna_host(w0), h1 = tf32_rna_host(w1);
          float* q = &b[(size_t)(off + (((int64_t)jt * K8 + kk) * 32 + lane) * 4)];
          q[0] = h0;
          q[1] = h1;
          q[2] = tf32_rna_host(w0 - h0);
          q[3] = tf32_rna_host(w1 - h1);
        }
    off += (int64_t)N8 * K8 * 8 * 8 * 2;
    for (int jj = 0; jj < no; ++jj) b[(size_t)(off + jj)] = net->params[poff + (int64_t)no * ni + jj];
    off += nn_tc_pad8(no);
    poff += (int64_t)ni * no + no;
  }
  return b;
}

// offset of layer l's W in lbm_mlp.params
int64_t off_of(const lbm_mlp* net, int l) {
  int64_t off = 0;
  for (int k = 0; k < l; ++k) off += (int64_t)net->sizes[k] * net->sizes[k + 1] + net->sizes[k + 1];
  return off;
}

lbm_status upload_net(lbm_sim* s, const lbm_mlp* net, int n_in, int64_t np) {
  for (int64_t k = 0; k < np; ++k)
    if (!std::isfinite(net->params[k])) return fail(LBM_ERR_ARG, "non-finite network parameter");
  const int64_t blob_n = (np + 2 * n_in + 3) / 4 * 4;
  std::vector<float> blob(blob_n, 0.f);
  int64_t off = 0;
  for (int l = 0; l < net->n_layers; ++l) {
    const int ni = net->sizes[l], no = net->sizes[l + 1];
    for (int j = 0; j < no; ++j)
      for (int k = 0; k < ni; ++k)
        blob[off + (int64_t)k * no + j] = net->params[off + (int64_t)j * ni + k];
    for (int j = 0; j < no; ++j) blob[off + (int64_t)ni * no + j] = net->params[off + (int64_t)ni * no + j];
    off += (int64_t)ni * no + no;
  }
  for (int k = 0; k < n_in; ++k) {
    blob[np + k] = net->in_mean ? net->in_mean[k] : 0.f;
    const float sd = net->in_std ? net->in_std[k] : 1.f;
    if (!(sd > 0.f) || !std::isfinite(sd)) return fail(LBM_ERR_ARG, "in_std must be > 0");
    if (!std::isfinite(blob[np + k])) return fail(LBM_ERR_ARG, "in_mean must be finite");
    blob[np + n_in + k] = sd;
  }
  // the CBC tuner's padded BF16 weights for the tensor-core path: per layer
  // [N_pad][K_pad], K_pad = 16 for the six inputs, hidden widths padded to a
  // multiple of 16, the last layer's N to 8; zeros in the padding
  std::vector<uint16_t> wb;
  if (n_in == 6) {
    int64_t woff = 0;
    for (int l = 0; l < net->n_layers; ++l) {
      const int ni = net->sizes[l], no = net->sizes[l + 1];
      const bool last = l == net->n_layers - 1;
      const int kp = l == 0 ? 16 : (ni + 15) / 16 * 16;
      const int npd = last ? 8 : (no + 15) / 16 * 16;
      wb.resize(wb.size() + (size_t)npd * kp, 0);
      for (int j = 0; j < no; ++j)
        for (int k = 0; k < ni; ++k)
          wb[(size_t)(woff + (int64_t)j * kp + k)] = bf16_rn(net->params[off_of(net, l) + (int64_t)j * ni + k]);
      woff += (int64_t)npd * kp;
    }
  }
  // the tensor-core blocks' blob (NN outflow: 81 inputs)
  std::vector<float> tcb;
  if (n_in == 81) tcb = nn_tc_blob(net);
  LBM_GUARD_BEGIN
  if (!s->nn.params_f || s->nn.blob_elems != (int32_t)blob_n ||
      s->nn.bf16_elems != (int64_t)wb.size() || s->nn.tc_elems != (int32_t)tcb.size()) {
    // all copies or none: a failed allocation leaves the current network
    const lbm_allocator* a = s->have_alloc ? &s->alloc : nullptr;
    const size_t bytes[4] = {blob.size() * sizeof(float), blob.size() * sizeof(double),
                             wb.size() * sizeof(uint16_t), tcb.size() * sizeof(float)};
    void* fresh[4] = {nullptr, nullptr, nullptr, nullptr};
    try {
      for (int k = 0; k < 4; ++k)
        if (bytes[k]) fresh[k] = lbm::dev_alloc_raw(a, bytes[k]);
    } catch (...) {
      for (void* q : fresh) lbm::dev_free_raw(a, q);
      throw;
    }
    if (s->nn.params_f) {
      // launch tables may still name the old copies: free them once the stream is idle
      lbm::sim_settle(s);
      ck(cudaStreamSynchronize(s->stream), "net sync");
      for (void* q : {(void*)s->nn.params_f, (void*)s->nn.params_d, (void*)s->nn.params_bf16,
                      (void*)s->nn.params_tc}) {
        if (!q) continue;
        s->owned.erase(std::remove(s->owned.begin(), s->owned.end(), q), s->owned.end());
        lbm::dev_free_raw(a, q);
      }
    }
    s->nn.params_f = (float*)fresh[0];
    s->nn.params_d = (double*)fresh[1];
    s->nn.params_bf16 = (uint16_t*)fresh[2];
    s->nn.params_tc = (float*)fresh[3];
    for (void* q : fresh)
      if (q) s->owned.push_back(q);
  }
  std::vector<double> blob_d(blob.begin(), blob.end());
  ck(cudaMemcpyAsync(s->nn.params_f, blob.data(), blob.size() * 4, cudaMemcpyHostToDevice,
                     s->stream), "net copy");
  ck(cudaMemcpyAsync(s->nn.params_d, blob_d.data(), blob_d.size() * 8, cudaMemcpyHostToDevice,
                     s->stream), "net copy");
  if (!wb.empty())
    ck(cudaMemcpyAsync(s->nn.params_bf16, wb.data(), wb.size() * 2, cudaMemcpyHostToDevice,
                       s->stream), "net copy");
  if (!tcb.empty())
    ck(cudaMemcpyAsync(s->nn.params_tc, tcb.data(), tcb.size() * 4, cudaMemcpyHostToDevice,
                       s->stream), "net copy");
  ck(cudaStreamSynchronize(s->stream), "net sync");
  s->nn.bf16_elems = (int64_t)wb.size();
  s->nn.tc_elems = (int32_t)tcb.size();
  s->nn.n_layers = net->n_layers;
  for (int l = 0; l <= LBM_MLP_MAX_LAYERS; ++l) s->nn.sizes[l] = l <= net->n_layers ? net->sizes[l] : 0;
  s->nn.act = net->act;
  s->nn.n_params = np;
  s->nn.blob_elems = (int32_t)blob_n;
  s->nn.out_scale = net->out_scale;
  return LBM_OK;
  LBM_GUARD_END
}

}  // namespace

namespace lbm {
void group_hold_flags(Group& g, bool hold);   // group.cu: test hook of the flag waits
}

extern "C" {

const char* lbm_last_error(void) { return g_err.c_str(); }

lbm_status lbm_set_default_allocator(const lbm_allocator* alloc) {
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(LBM_ERR_ARG, "allocator needs both alloc and free");
  lbm::set_default_allocator(alloc);
  return LBM_OK;
}

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
  if (cfg->layout != LBM_LAYOUT_AB && cfg->layout != LBM_LAYOUT_AA)
    return fail(LBM_ERR_ARG, "unknown layout");
  if ((int64_t)9 * cfg->ny * (((int64_t)cfg->nx + 2 + 63) / 64 * 64) >= ((int64_t)1 << 31))
    return fail(LBM_ERR_ARG, "9 * ny * pitch must stay below 2^31 elements");
  if (!(cfg->tau > 0.5) || !std::isfinite(cfg->tau)) return fail(LBM_ERR_ARG, "tau must be > 1/2");
  if (cfg->collision != LBM_BGK && cfg->collision != LBM_MRT)
    return fail(LBM_ERR_ARG, "unknown collision");
  if (cfg->precision < LBM_FP64 || cfg->precision > LBM_FP16DEV)
    return fail(LBM_ERR_ARG, "unknown precision");
  if (!(std::fabs(cfg->u_in) < 1.0)) return fail(LBM_ERR_ARG, "|u_in| must be < 1");
  if (!(cfg->rho_out > 0.0)) return fail(LBM_ERR_ARG, "rho_out must be > 0");
  if (cfg->force_capacity < 0) return fail(LBM_ERR_ARG, "force_capacity must be >= 0");
  if (cfg->ramp_steps < 0) return fail(LBM_ERR_ARG, "ramp_steps must be >= 0");
  if (cfg->alloc && (!cfg->alloc->alloc || !cfg->alloc->free))
    return fail(LBM_ERR_ARG, "allocator needs both alloc and free");
  if (!lbm::mrt_rates_valid(*cfg)) return fail(LBM_ERR_ARG, "MRT rates must lie in [0, 2)");

  lbm_sim* s = new (std::nothrow) lbm_sim();
  if (!s) return fail(LBM_ERR_OOM, "host allocation failed");
  LBM_GUARD_BEGIN
  s->cfg = *cfg;
  s->nx = cfg->nx;
  s->ny = cfg->ny;
  s->prec = cfg->precision;
  s->elem = s->prec == LBM_FP64 ? 8 : (s->prec == LBM_FP32 ? 4 : 2);
  s->layout = cfg->layout;
  // the in-place layout keeps a ghost column on each side (x = -1 and x = nx)
  s->pitch = ((int64_t)s->nx + (s->layout == LBM_LAYOUT_AA ? 2 : 0) + 63) / 64 * 64;
  s->plane = s->pitch * s->ny;
  s->rho_out = cfg->rho_out;
  if (cfg->alloc) {
    s->alloc = *cfg->alloc;
    s->have_alloc = true;
  } else {
    s->have_alloc = lbm::default_allocator(&s->alloc);
  }
  s->cfg.alloc = nullptr;
  if (cfg->stream) {
    s->stream = (cudaStream_t)cfg->stream;
  } else {
    ck(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    s->own_stream = true;
  }
  // + slack: the staged kernel copies whole 16-byte aligned row segments that
  // may run up to 128 + 8 elements past the last row of the last population
  const size_t bytes = ((size_t)9 * s->plane + 256) * s->elem;
  if (s->layout == LBM_LAYOUT_AA) {
    s->buf_alloc = dev_alloc(s, bytes);
    s->buf[0] = static_cast<unsigned char*>(s->buf_alloc) + s->elem;   // x = -1 at the start
    s->buf[1] = s->buf[0];
  } else {
    s->buf[0] = dev_alloc(s, bytes);
    s->buf[1] = dev_alloc(s, bytes);
    if (s->prec == LBM_FP16DEV) make_tensor_maps(s);   // row windows of the staged kernel
  }
  const int64_t cells = (int64_t)s->nx * s->ny;
  s->kind = (uint8_t*)dev_alloc(s, cells);
  s->words_per_row = (s->nx + 127) / 128 * 4;   // whole 16-byte groups per row
  s->solid_bits = (uint32_t*)dev_alloc(s, (size_t)s->words_per_row * s->ny * 4);
  s->links = (uint8_t*)dev_alloc(s, cells);
  s->near_bits = (uint32_t*)dev_alloc(s, (size_t)s->words_per_row * s->ny * 4);
  s->ring_auto = cfg->force_capacity == 0;
  s->ring_cap = s->ring_auto ? kInitialRing : cfg->force_capacity;
  s->ring = (double*)dev_alloc(s, (size_t)2 * s->ring_cap * sizeof(double));
  s->status = (int*)dev_alloc(s, sizeof(int));
  s->scratch_sums = (double*)dev_alloc(s, ((size_t)s->ny + 1) * sizeof(double));
  s->nn_fallbacks = (unsigned long long*)dev_alloc(s, sizeof(unsigned long long));
  ck(cudaMemsetAsync(s->kind, 0, cells, s->stream), "memset");
  ck(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream), "memset");
  ck(cudaMemsetAsync(s->nn_fallbacks, 0, sizeof(unsigned long long), s->stream), "memset");
  ck(cudaMemsetAsync(s->ring, 0, (size_t)2 * s->ring_cap * sizeof(double), s->stream), "memset");
  // padding (and ghost) columns are never read by the step, but keep them defined
  if (s->layout == LBM_LAYOUT_AA) {
    ck(cudaMemsetAsync(s->buf_alloc, 0, bytes, s->stream), "memset");
  } else {
    ck(cudaMemsetAsync(s->buf[0], 0, bytes, s->stream), "memset");
    ck(cudaMemsetAsync(s->buf[1], 0, bytes, s->stream), "memset");
  }
  lbm::launch_geometry_prep(s->kind, s->nx, s->ny, s->cfg.x_periodic, s->solid_bits,
                            s->words_per_row, s->links, s->near_bits, s->stream);
  lbm::launch_init_equilibrium(s->prec, s->buf[0], s->nx, s->ny, s->pitch, s->plane, nullptr,
                               nullptr, nullptr, s->stream, lbm::pop_map(s, 0));
  ck(cudaGetLastError(), "init launch");
  lbm::group_init(s->own, std::vector<lbm_sim*>{s}, true);
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
  if (s->batch_refs > 0) return fail(LBM_ERR_STATE, "destroy the batches holding this sim first");
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
  {
    const int tiles = (s->nx + 127) / 128;
    s->solid_tile_rows.assign((size_t)tiles * s->ny, 0);
    for (int y = 0; y < s->ny; ++y)
      for (int x = 0; x < s->nx; ++x)
        if (kind[(int64_t)y * s->nx + x] == LBM_CELL_SOLID)
          s->solid_tile_rows[(size_t)y * tiles + x / 128] = 1;
  }
  LBM_GUARD_BEGIN
  ck(cudaMemcpyAsync(s->kind, kind, cells, cudaMemcpyHostToDevice, s->stream), "kind copy");
  lbm::launch_geometry_prep(s->kind, s->nx, s->ny, s->cfg.x_periodic, s->solid_bits,
                            s->words_per_row, s->links, s->near_bits, s->stream);
  ck(cudaGetLastError(), "geometry launch");
  ck(cudaStreamSynchronize(s->stream), "geometry sync");
  s->version++;
  return LBM_OK;
  LBM_GUARD_END
}

static void reset_counters(lbm_sim* s) {
  lbm::sim_settle(s);
  s->last_group = nullptr;
  ck(cudaMemsetAsync(s->status, 0, sizeof(int), s->stream), "memset");
  ck(cudaMemsetAsync(s->nn_fallbacks, 0, sizeof(unsigned long long), s->stream), "memset");
  s->t_host = 0;
  s->drained = 0;
}

lbm_status lbm_init_equilibrium(lbm_sim* s, const double* rho, const double* ux, const double* uy) {
  if (lbm_status st = check_sim(s)) return st;
  LBM_GUARD_BEGIN
  s->cur = 0;
  if (!rho && !ux && !uy) {
    lbm::launch_init_equilibrium(s->prec, s->buf[0], s->nx, s->ny, s->pitch, s->plane, nullptr,
                                 nullptr, nullptr, s->stream, lbm::pop_map(s, 0));
    ck(cudaGetLastError(), "init launch");
  } else {
    // the fields stream through the scratch in chunks of whole rows
    int rows = 0;
    double* d = field_scratch(s, 3, &rows);
    const size_t nx = (size_t)s->nx;
    for (int y0 = 0; y0 < s->ny; y0 += rows) {
      const int r = std::min(rows, s->ny - y0);
      const size_t n = (size_t)r * nx;
      const double* src[3] = {rho, ux, uy};
      const double* dev[3] = {nullptr, nullptr, nullptr};
      for (int k = 0; k < 3; ++k) {
        if (!src[k]) continue;
        ck(cudaMemcpyAsync(d + k * n, src[k] + (size_t)y0 * nx, n * 8, cudaMemcpyHostToDevice,
                           s->stream), "field copy");
        dev[k] = d + k * n;
      }
      lbm::launch_init_equilibrium(s->prec, s->buf[0], s->nx, s->ny, s->pitch, s->plane, dev[0],
                                   dev[1], dev[2], s->stream, lbm::pop_map(s, 0), y0, r);
      ck(cudaGetLastError(), "init launch");
    }
  }
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
  s->version++;
  return LBM_OK;
}

lbm_status lbm_set_outflow_nn(lbm_sim* s, const lbm_mlp* net, double fallback_drho) {
  if (lbm_status st = check_sim(s)) return st;
  if (s->layout == LBM_LAYOUT_AA)
    return fail(LBM_ERR_UNSUPPORTED, "the in-place (AA) layout supports the Zou & He outflow only");
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
  if (lbm_status st = upload_net(s, net, 81, np)) return st;
  s->nn_drho = fallback_drho;
  s->east = lbm::EAST_EXTERNAL;
  s->outflow = LBM_OUTFLOW_NN;
  s->version++;
  return LBM_OK;
}

lbm_status lbm_set_outflow_cbc(lbm_sim* s, double sigma, double kappa2, double mach, double length,
                               const lbm_mlp* tuner, int32_t exact_mass) {
  if (lbm_status st = check_sim(s)) return st;
  if (s->layout == LBM_LAYOUT_AA)
    return fail(LBM_ERR_UNSUPPORTED, "the in-place (AA) layout supports the Zou & He outflow only");
  if (s->cfg.x_periodic) return fail(LBM_ERR_STATE, "x is periodic: there is no outflow");
  if (s->nx < 4) return fail(LBM_ERR_ARG, "the characteristic outflow needs nx >= 4");
  if (!(sigma >= 0.0) || !std::isfinite(sigma)) return fail(LBM_ERR_ARG, "sigma must be >= 0");
  if (!std::isfinite(kappa2)) return fail(LBM_ERR_ARG, "kappa2 must be finite");
  if (!(std::fabs(mach) < 1.0)) return fail(LBM_ERR_ARG, "|mach| must be < 1");
  if (!(length >= 0.0) || !std::isfinite(length)) return fail(LBM_ERR_ARG, "length must be >= 0");
  if (exact_mass != 0 && exact_mass != 1) return fail(LBM_ERR_ARG, "exact_mass must be 0 or 1");
  if (tuner) {
    if (!tuner->params) return fail(LBM_ERR_ARG, "tuner->params is NULL");
    if (tuner->n_layers < 1 || tuner->n_layers > 3)
      return fail(LBM_ERR_ARG, "the tuner has 1..3 layers");
    if (tuner->sizes[0] != 6 || tuner->sizes[tuner->n_layers] < 1 ||
        tuner->sizes[tuner->n_layers] > 2)
      return fail(LBM_ERR_ARG, "the tuner maps 6 inputs to 1 or 2 outputs");
    int64_t np = 0;
    for (int l = 0; l < tuner->n_layers; ++l) {
      if (tuner->sizes[l + 1] < 1 || tuner->sizes[l + 1] > 32)
        return fail(LBM_ERR_ARG, "tuner layers must have 1..32 units");
      np += (int64_t)tuner->sizes[l] * tuner->sizes[l + 1] + tuner->sizes[l + 1];
    }
    if (tuner->n_params != np) return fail(LBM_ERR_ARG, "n_params does not match the layer sizes");
    if (tuner->act != 0 && tuner->act != 1)
      return fail(LBM_ERR_ARG, "act must be 0 (tanh) or 1 (leaky)");
    if (lbm_status st = upload_net(s, tuner, 6, np)) return st;
  } else {
    s->nn.n_layers = 0;
  }
  s->cbc_sigma = sigma;
  s->cbc_kappa2 = kappa2;
  s->cbc_mach = mach;
  s->cbc_length = length;
  s->cbc_exact = exact_mass;
  s->east = lbm::EAST_EXTERNAL;
  s->outflow = LBM_OUTFLOW_CBC;
  s->version++;
  return LBM_OK;
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

// ---- training rows and training (Sec. 3.1) ---------------------------------

lbm_status lbm_capture_plane(lbm_sim* s, int32_t x_t, int32_t every, float* dev_rows,
                             int64_t cap_rows) {
  if (lbm_status st = check_sim(s)) return st;
  if (s->layout == LBM_LAYOUT_AA)
    return fail(LBM_ERR_UNSUPPORTED, "capture needs the two-buffer (AB) layout");
  if (!dev_rows) {
    s->cap_every = 0;
    s->cap_out = nullptr;
    s->cap_capacity = 0;
    s->cap_rows = 0;
    return LBM_OK;
  }
  if (x_t < 4 || x_t > s->nx - 2) return fail(LBM_ERR_ARG, "x_t must be in [4, nx-2]");
  if (every < 1) return fail(LBM_ERR_ARG, "every must be >= 1");
  if (cap_rows < 0) return fail(LBM_ERR_ARG, "cap_rows must be >= 0");
  s->cap_x = x_t;
  s->cap_every = every;
  s->cap_out = dev_rows;
  s->cap_capacity = cap_rows;
  s->cap_rows = 0;
  return LBM_OK;
}

lbm_status lbm_capture_snapshot(lbm_sim* s, int32_t x_begin, int32_t x_end, float* dev_rows) {
  if (lbm_status st = check_sim(s)) return st;
  if (s->layout == LBM_LAYOUT_AA)
    return fail(LBM_ERR_UNSUPPORTED, "capture needs the two-buffer (AB) layout");
  if (!dev_rows) return fail(LBM_ERR_ARG, "dev_rows is NULL");
  if (!s->solid_bits) return fail(LBM_ERR_STATE, "set the geometry first");
  if (x_begin < 4 || x_end <= x_begin || x_end > s->nx - 1)
    return fail(LBM_ERR_ARG, "columns must satisfy 4 <= x_begin < x_end <= nx-1");
  if ((int64_t)(x_end - x_begin) > 65535) return fail(LBM_ERR_ARG, "at most 65535 columns");
  LBM_GUARD_BEGIN
  lbm::CaptureParams c{};
  c.src = s->buf[s->cur];
  c.solid_bits = s->solid_bits;
  c.words_per_row = s->words_per_row;
  c.nx = s->nx;
  c.ny = s->ny;
  c.pitch = s->pitch;
  c.plane = s->plane;
  c.x_t = x_begin;
  c.out = dev_rows;
  lbm::launch_snapshot(s->prec, c, x_end - x_begin, s->stream);
  ck(cudaGetLastError(), "snapshot launch");
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_capture_count(lbm_sim* s, int64_t* rows) {
  if (lbm_status st = check_sim(s)) return st;
  if (!rows) return fail(LBM_ERR_ARG, "rows is NULL");
  *rows = s->cap_rows;
  return LBM_OK;
}


lbm_status lbm_train_opts_default(lbm_train_opts* o) {
  if (!o) return fail(LBM_ERR_ARG, "opts is NULL");
  *o = lbm_train_opts{};
  o->lr = 1e-5;
  o->beta1 = 0.9;
  o->beta2 = 0.999;
  o->eps = 1e-8;
  return LBM_OK;
}

lbm_status lbm_nn_dataset_stats(const float* rows, int64_t n, void* stream, float* in_mean,
                                float* in_std, float* out_scale) {
  if (!rows || !in_mean || !in_std || !out_scale) return fail(LBM_ERR_ARG, "NULL argument");
  if (n < 1) return fail(LBM_ERR_ARG, "n_rows must be >= 1");
  LBM_GUARD_BEGIN
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nd = lbm::dataset_stats_scratch_doubles();
  DevBuf scratch(nd * sizeof(double));
  lbm::dataset_stats(rows, n, scratch.as<double>(), st);
  ck(cudaGetLastError(), "stats launch");
  std::vector<double> mv(164);
  ck(cudaMemcpyAsync(mv.data(), scratch.as<double>() + (nd - 164), 164 * sizeof(double),
                     cudaMemcpyDeviceToHost, st), "stats copy");
  ck(cudaStreamSynchronize(st), "stats sync");
  constexpr double kMinStd = 1e-12;
  for (int c = 0; c < 81; ++c) {
    in_mean[c] = (float)mv[c];
    const double sd = std::sqrt(mv[82 + c]);
    in_std[c] = (float)(sd < kMinStd ? 1.0 : sd);
  }
  const double rs = std::sqrt(mv[82 + 81]);
  *out_scale = (float)(rs < kMinStd ? 1.0 : rs);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_nn_train(const float* rows, int64_t n_rows, const int32_t* order, int64_t n_steps,
                        const lbm_train_opts* opts, const lbm_mlp* net, float* params_out,
                        float* adam_m, float* adam_v, double* loss_log) {
  if (!params_out) return fail(LBM_ERR_ARG, "params_out is NULL");
  return run_training(rows, n_rows, order, n_steps, opts, net, 0, params_out, adam_m, adam_v,
                      loss_log, nullptr);
}

lbm_status lbm_nn_loss_grad(const float* rows, int64_t n_rows, const int32_t* order,
                            int64_t n_batches, const lbm_train_opts* opts, const lbm_mlp* net,
                            double* losses, float* grads) {
  if (!losses) return fail(LBM_ERR_ARG, "losses is NULL");
  return run_training(rows, n_rows, order, n_batches, opts, net, grads ? 1 : 2, nullptr, nullptr,
                      nullptr, losses, grads);
}

lbm_status lbm_step(lbm_sim* s, int64_t n) {
  if (lbm_status st = check_sim(s)) return st;
  if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
  LBM_GUARD_BEGIN
  lbm::group_step(s->own, n);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_sync(lbm_sim* s) {
  if (lbm_status st = check_sim(s)) return st;
  LBM_GUARD_BEGIN
  lbm::sim_settle(s);
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
  lbm::sim_settle(s);
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
  LBM_GUARD_BEGIN
  int rows = 0;
  double* d = field_scratch(s, 3, &rows);
  const size_t nx = (size_t)s->nx;
  for (int y0 = 0; y0 < s->ny; y0 += rows) {
    const int r = std::min(rows, s->ny - y0);
    const size_t n = (size_t)r * nx;
    lbm::launch_export(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane, nullptr, d,
                       d + n, d + 2 * n, s->stream, lbm::pop_map(s, s->t_host), y0, r);
    ck(cudaGetLastError(), "export launch");
    double* dst[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k)
      if (dst[k])
        ck(cudaMemcpyAsync(dst[k] + (size_t)y0 * nx, d + k * n, n * 8, cudaMemcpyDeviceToHost,
                           s->stream), "field copy");
  }
  return read_status(s);
  LBM_GUARD_END
}

lbm_status lbm_get_populations(lbm_sim* s, double* f) {
  if (lbm_status st = check_sim(s)) return st;
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  const size_t cells = (size_t)s->nx * s->ny;
  LBM_GUARD_BEGIN
  int rows = 0;
  double* d = field_scratch(s, 9, &rows);
  const size_t nx = (size_t)s->nx;
  for (int y0 = 0; y0 < s->ny; y0 += rows) {
    const int r = std::min(rows, s->ny - y0);
    const size_t n = (size_t)r * nx;
    lbm::launch_export(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane, d, nullptr,
                       nullptr, nullptr, s->stream, lbm::pop_map(s, s->t_host), y0, r);
    ck(cudaGetLastError(), "export launch");
    // nine planes of r rows into the host planes of ny rows
    ck(cudaMemcpy2DAsync(f + (size_t)y0 * nx, cells * 8, d, n * 8, n * 8, 9,
                         cudaMemcpyDeviceToHost, s->stream), "population copy");
  }
  return read_status(s);
  LBM_GUARD_END
}

lbm_status lbm_set_populations(lbm_sim* s, const double* f) {
  if (lbm_status st = check_sim(s)) return st;
  if (!f) return fail(LBM_ERR_ARG, "f is NULL");
  const size_t cells = (size_t)s->nx * s->ny;
  LBM_GUARD_BEGIN
  int rows = 0;
  double* d = field_scratch(s, 9, &rows);
  const size_t nx = (size_t)s->nx;
  for (int y0 = 0; y0 < s->ny; y0 += rows) {
    const int r = std::min(rows, s->ny - y0);
    const size_t n = (size_t)r * nx;
    ck(cudaMemcpy2DAsync(d, n * 8, f + (size_t)y0 * nx, cells * 8, n * 8, 9,
                         cudaMemcpyHostToDevice, s->stream), "population copy");
    lbm::launch_import(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane, d, s->stream,
                       lbm::pop_map(s, s->t_host), y0, r);
    ck(cudaGetLastError(), "import launch");
  }
  ck(cudaStreamSynchronize(s->stream), "sync");
  return LBM_OK;
  LBM_GUARD_END
}

// ---- checkpoints ------------------------------------------------------------
namespace {
struct CheckpointHeader {
  char magic[8];
  int32_t nx, ny, precision, pad;
  int64_t t, elems;
};
constexpr char kCheckpointMagic[8] = {'G', 'B', '3', 'L', 'B', 'M', 'v', '1'};
}  // namespace

lbm_status lbm_save(lbm_sim* s, const char* path) {
  if (lbm_status st = check_sim(s)) return st;
  if (!path) return fail(LBM_ERR_ARG, "path is NULL");
  LBM_GUARD_BEGIN
  lbm::sim_settle(s);
  const bool aa = s->layout == LBM_LAYOUT_AA;
  const int64_t elems = 9 * s->plane + (aa ? 1 : 0);
  std::vector<unsigned char> host((size_t)(elems * (int64_t)s->elem));
  ck(cudaMemcpyAsync(host.data(), aa ? s->buf_alloc : s->buf[s->cur], host.size(),
                     cudaMemcpyDeviceToHost, s->stream), "checkpoint copy");
  if (lbm_status st = read_status(s)) return st;
  CheckpointHeader h{};
  memcpy(h.magic, kCheckpointMagic, 8);
  h.nx = s->nx;
  h.ny = s->ny;
  h.precision = s->prec;
  h.pad = s->layout;
  h.t = s->t_host;
  h.elems = elems;
  FILE* fp = fopen(path, "wb");
  if (!fp) return fail(LBM_ERR_ARG, std::string("cannot open ") + path + " for writing");
  const bool ok = fwrite(&h, sizeof(h), 1, fp) == 1 &&
                  fwrite(host.data(), 1, host.size(), fp) == host.size();
  if (fclose(fp) != 0 || !ok) return fail(LBM_ERR_ARG, std::string("write to ") + path + " failed");
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_load(lbm_sim* s, const char* path) {
  if (lbm_status st = check_sim(s)) return st;
  if (!path) return fail(LBM_ERR_ARG, "path is NULL");
  FILE* fp = fopen(path, "rb");
  if (!fp) return fail(LBM_ERR_ARG, std::string("cannot open ") + path);
  CheckpointHeader h{};
  const bool hdr = fread(&h, sizeof(h), 1, fp) == 1;
  if (!hdr || memcmp(h.magic, kCheckpointMagic, 8) != 0) {
    fclose(fp);
    return fail(LBM_ERR_ARG, "not a checkpoint of this library");
  }
  const bool aa = s->layout == LBM_LAYOUT_AA;
  if (h.nx != s->nx || h.ny != s->ny || h.precision != s->prec || h.pad != s->layout ||
      h.elems != 9 * s->plane + (aa ? 1 : 0) || h.t < 0) {
    fclose(fp);
    return fail(LBM_ERR_ARG, "the checkpoint is for another lattice size, precision or layout");
  }
  std::vector<unsigned char> host((size_t)(h.elems * (int64_t)s->elem));
  const bool body = fread(host.data(), 1, host.size(), fp) == host.size();
  fclose(fp);
  if (!body) return fail(LBM_ERR_ARG, "the checkpoint is truncated");
  LBM_GUARD_BEGIN
  reset_counters(s);
  ck(cudaMemcpyAsync(aa ? s->buf_alloc : s->buf[0], host.data(), host.size(),
                     cudaMemcpyHostToDevice, s->stream), "checkpoint copy");
  ck(cudaStreamSynchronize(s->stream), "checkpoint sync");
  s->cur = 0;
  s->t_host = h.t;
  s->drained = h.t;
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_mass(lbm_sim* s, double* mass) {
  if (lbm_status st = check_sim(s)) return st;
  if (!mass) return fail(LBM_ERR_ARG, "mass is NULL");
  LBM_GUARD_BEGIN
  lbm::launch_mass(s->prec, s->buf[s->cur], s->nx, s->ny, s->pitch, s->plane, s->scratch_sums,
                   s->ny, s->scratch_sums + s->ny, s->stream, lbm::pop_map(s, s->t_host));
  ck(cudaGetLastError(), "mass launch");
  ck(cudaMemcpyAsync(mass, s->scratch_sums + s->ny, 8, cudaMemcpyDeviceToHost, s->stream), "copy");
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

static lbm_status check_tiling(int32_t rows, int32_t variant) {
  if (rows < 1 || rows > 4096) return fail(LBM_ERR_ARG, "rows must be in 1..4096");
  if (variant < 0 || variant >= lbm::step_variants()) return fail(LBM_ERR_ARG, "bad variant");
  if (lbm::step_variant_is_bulk(variant) && rows < 2)
    return fail(LBM_ERR_ARG, "the staged variants need rows >= 2");
  return LBM_OK;
}

lbm_status lbm_set_tiling(lbm_sim* s, int32_t rows, int32_t variant) {
  if (lbm_status st = check_sim(s)) return st;
  if (lbm_status st = check_tiling(rows, variant)) return st;
  if (s->layout == LBM_LAYOUT_AA && lbm::step_variant_is_bulk(variant) && variant != 3)
    return fail(LBM_ERR_UNSUPPORTED, "the in-place (AA) layout runs on variants 0-3");
  LBM_GUARD_BEGIN
  lbm::group_set_tiling(s->own, rows, variant);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_debug_hold_dataflow(lbm_sim* s, int32_t hold) {
  if (lbm_status st = check_sim(s)) return st;
  if (!lbm::step_variant_dataflow(s->own.variant))
    return fail(LBM_ERR_STATE, "the sim's tiling is not the dataflow variant (6)");
  LBM_GUARD_BEGIN
  lbm::group_hold_flags(s->own, hold != 0);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_get_tiling(lbm_sim* s, int32_t* rows, int32_t* variant) {
  if (lbm_status st = check_sim(s)) return st;
  if (!rows || !variant) return fail(LBM_ERR_ARG, "outputs must be non-NULL");
  *rows = s->own.rows;
  *variant = s->own.variant;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_sim* s, int32_t steps, int64_t flush_bytes, float* best_ms) {
  if (lbm_status st = check_sim(s)) return st;
  if (steps < 1 || steps > 10000) return fail(LBM_ERR_ARG, "steps must be in 1..10000");
  if (flush_bytes < 0) return fail(LBM_ERR_ARG, "flush_bytes must be >= 0");
  LBM_GUARD_BEGIN
  const float ms = lbm::group_autotune(s->own, steps, flush_bytes);
  if (best_ms) *best_ms = ms;
  return LBM_OK;
  LBM_GUARD_END
}

// ---- batches -------------------------------------------------------------------
lbm_status lbm_batch_create(lbm_sim* const* sims, int32_t n, lbm_batch** out) {
  if (!sims || !out || n < 1) return fail(LBM_ERR_ARG, "sims and out must be non-NULL, n >= 1");
  *out = nullptr;
  for (int32_t k = 0; k < n; ++k) {
    if (lbm_status st = check_sim(sims[k])) return st;
    if (sims[k]->layout == LBM_LAYOUT_AA)
      return fail(LBM_ERR_UNSUPPORTED, "an in-place (AA) lattice runs alone, not in a batch");
    if (sims[k]->prec != sims[0]->prec)
      return fail(LBM_ERR_ARG, "batch members must share one precision");
    if (sims[k]->stream != sims[0]->stream)
      return fail(LBM_ERR_ARG, "batch members must share one stream (lbm_config.stream)");
    if (sims[k]->t_host != sims[0]->t_host || sims[k]->cur != sims[0]->cur)
      return fail(LBM_ERR_STATE, "batch members must be at the same step");
    for (int32_t j = 0; j < k; ++j)
      if (sims[j] == sims[k]) return fail(LBM_ERR_ARG, "a sim appears twice in the batch");
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return fail(LBM_ERR_OOM, "host allocation failed");
  try {
    for (int32_t k = 0; k < n; ++k) lbm::sim_settle(sims[k]);
    lbm::group_init(b->g, std::vector<lbm_sim*>(sims, sims + n), false);
    b->g.rows = 8;
    b->g.variant = 1;
    ck(cudaStreamSynchronize(b->g.stream), "batch sync");
    for (int32_t k = 0; k < n; ++k) sims[k]->batch_refs++;
    *out = b;
    return LBM_OK;
  } catch (const CudaError& ce) {
    lbm::group_release(b->g);
    delete b;
    return from_cuda(ce);
  } catch (...) {
    lbm::group_release(b->g);
    delete b;
    return fail(LBM_ERR_OOM, "allocation failed");
  }
}

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  LBM_GUARD_BEGIN
  lbm::group_finalize(b->g);
  for (lbm_sim* s : b->g.sims) s->batch_refs--;
  lbm::group_release(b->g);
  delete b;
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t n) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  if (n < 0) return fail(LBM_ERR_ARG, "n must be >= 0");
  for (const lbm_sim* s : b->g.sims)
    if (s->t_host != b->g.sims[0]->t_host || s->cur != b->g.sims[0]->cur)
      return fail(LBM_ERR_STATE, "batch members were stepped apart: not in lockstep");
  LBM_GUARD_BEGIN
  lbm::group_step(b->g, n);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_batch_sync(lbm_batch* b) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  LBM_GUARD_BEGIN
  lbm::group_finalize(b->g);
  lbm_status worst = LBM_OK;
  for (lbm_sim* s : b->g.sims) {
    const lbm_status st = read_status(s);
    if (st != LBM_OK && worst == LBM_OK) worst = st;
  }
  return worst;
  LBM_GUARD_END
}

lbm_status lbm_batch_set_tiling(lbm_batch* b, int32_t rows, int32_t variant) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  if (lbm_status st = check_tiling(rows, variant)) return st;
  LBM_GUARD_BEGIN
  lbm::group_set_tiling(b->g, rows, variant);
  return LBM_OK;
  LBM_GUARD_END
}

lbm_status lbm_batch_get_tiling(lbm_batch* b, int32_t* rows, int32_t* variant) {
  if (!b || !rows || !variant) return fail(LBM_ERR_ARG, "arguments must be non-NULL");
  *rows = b->g.rows;
  *variant = b->g.variant;
  return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t steps, int64_t flush_bytes, float* best_ms) {
  if (!b) return fail(LBM_ERR_ARG, "batch is NULL");
  if (steps < 1 || steps > 10000) return fail(LBM_ERR_ARG, "steps must be in 1..10000");
  if (flush_bytes < 0) return fail(LBM_ERR_ARG, "flush_bytes must be >= 0");
  LBM_GUARD_BEGIN
  const float ms = lbm::group_autotune(b->g, steps, flush_bytes);
  if (best_ms) *best_ms = ms;
  return LBM_OK;
  LBM_GUARD_END
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
