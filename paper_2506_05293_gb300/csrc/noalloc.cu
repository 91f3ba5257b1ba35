// lbm_step_noalloc: one FP32 time step on caller-owned device buffers that
// performs no device allocation at all.
//
// Some callers cannot allocate device memory: code running inside a CUDA
// stream capture that must not add allocation nodes, host frameworks that own
// every byte of device memory through their own pool, or real-time loops that
// forbid allocator calls after start-up.  They can still step a lattice they
// allocated themselves through this entry point.
//
// It is a variant of the fused step kernel (step.cu): same pull streaming,
// full-way bounce-back, Zou & He inlet/outflow and BGK/MRT collision, but it
// reads the cell kinds directly (no prepared solid mask or link table) and
// sums the momentum-exchange force through per-block FP64 partials kept in a
// file-scope device array instead of library-allocated scratch.  One block
// handles one strip of 128 columns x 8 rows, so the array bounds the lattice
// size: at most kMaxStrips strips (8,388,608 nodes).
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lattice.cuh"
#include "sim.cuh"

namespace lbm {
namespace {

constexpr int kRows = 8;           // rows per strip (one strip = one block)
constexpr int kMaxStrips = 8192;   // strips the scratch array can hold
constexpr int kMaxDevices = 64;

// Force partials (F_x, F_y) of every block of the last call, 128 KiB.  Every
// call writes each slot it later reads, so nothing needs clearing between
// calls; calls that overlap on the GPU (different streams) race on it.
static __device__ __align__(256) double g_noalloc_partials[2 * kMaxStrips];

struct NoAllocParams {
  const float* src;
  float* dst;
  const uint8_t* kind;
  int nx, ny, pitch, plane;
  float omega, u_in, rho_out;
  MrtRates<float> mrt;
  double v_amp, u_in_d;
  int64_t ramp_steps;
  uint64_t seed;
  int x_periodic, coll;
  int64_t t;
  double* partials;
  double* force;
};

__global__ void __launch_bounds__(128) noalloc_step_kernel(const NoAllocParams p) {
  const int tiles_x = (p.nx + 127) >> 7;
  const int strip = blockIdx.x;
  const int x = (strip % tiles_x) * 128 + threadIdx.x;
  const int y0 = (strip / tiles_x) * kRows;
  const int y1 = min(y0 + kRows, p.ny);
  double fx = 0.0, fy = 0.0;
  if (x < p.nx) {
    const int xm = x == 0 ? p.nx - 1 : x - 1;
    const int xp = x == p.nx - 1 ? 0 : x + 1;
    const bool west = !p.x_periodic && x == 0;
    const bool east = !p.x_periodic && x == p.nx - 1;
    for (int y = y0; y < y1; ++y) {
      const int ym = y == 0 ? p.ny - 1 : y - 1;
      const int yp = y == p.ny - 1 ? 0 : y + 1;
      const int rc = y * p.pitch, rm = ym * p.pitch, rp = yp * p.pitch;
      float h[9];
      h[0] = p.src[rc + x];
      h[1] = p.src[1 * p.plane + rc + xm];
      h[2] = p.src[2 * p.plane + rm + x];
      h[3] = p.src[3 * p.plane + rc + xp];
      h[4] = p.src[4 * p.plane + rp + x];
      h[5] = p.src[5 * p.plane + rm + xm];
      h[6] = p.src[6 * p.plane + rm + xp];
      h[7] = p.src[7 * p.plane + rp + xp];
      h[8] = p.src[8 * p.plane + rp + xm];
      const int o = rc + x;
      const uint8_t k = p.kind[(int64_t)y * p.nx + x];
      if (k != LBM_CELL_FLUID) {
        if (k == LBM_CELL_SOLID) {
          // momentum exchange over links to fluid neighbours s - c_i
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            int sx = x - cx(i);
            int sy = y - cy(i);
            sy = sy < 0 ? sy + p.ny : (sy >= p.ny ? sy - p.ny : sy);
            if (sx < 0 || sx >= p.nx) {
              if (!p.x_periodic) continue;
              sx = sx < 0 ? sx + p.nx : sx - p.nx;
            }
            if (p.kind[(int64_t)sy * p.nx + sx] != LBM_CELL_FLUID) continue;
            const double v = (double)h[i] + (double)p.src[opp(i) * p.plane + o] +
                             2.0 * wgt<double>(i);
            fx += cx(i) * v;
            fy += cy(i) * v;
          }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) p.dst[i * p.plane + o] = h[opp(i)];
        continue;
      }
      if (west) {
        const float v = (float)inlet_perturbation(p.seed, p.t, y, p.v_amp);
        const float u =
            p.ramp_steps > 0 ? (float)inlet_velocity(p.u_in_d, p.ramp_steps, p.t) : p.u_in;
        zouhe_west<float>(h, u, v);
      } else if (east) {
        zouhe_east<float>(h, p.rho_out);
      }
      float drho, ux, uy;
      if (p.coll == LBM_BGK)
        collide_bgk<float>(h, p.omega, drho, ux, uy);
      else
        collide_mrt<float>(h, p.mrt, drho, ux, uy);
#pragma unroll
      for (int i = 0; i < 9; ++i) p.dst[i * p.plane + o] = h[i];
    }
  }
  // fixed-order block sum of the force partial
  __shared__ double s_x[4], s_y[4];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    fx += __shfl_down_sync(0xffffffffu, fx, off);
    fy += __shfl_down_sync(0xffffffffu, fy, off);
  }
  if ((threadIdx.x & 31) == 0) {
    s_x[threadIdx.x >> 5] = fx;
    s_y[threadIdx.x >> 5] = fy;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    p.partials[2 * strip] = (s_x[0] + s_x[1]) + (s_x[2] + s_x[3]);
    p.partials[2 * strip + 1] = (s_y[0] + s_y[1]) + (s_y[2] + s_y[3]);
  }
}

__global__ void noalloc_reduce_kernel(const double* partials, int n, double* force) {
  __shared__ double s_x[4], s_y[4];
  double ax = 0.0, ay = 0.0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    ax += partials[2 * b];
    ay += partials[2 * b + 1];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ax += __shfl_down_sync(0xffffffffu, ax, off);
    ay += __shfl_down_sync(0xffffffffu, ay, off);
  }
  if ((threadIdx.x & 31) == 0) {
    s_x[threadIdx.x >> 5] = ax;
    s_y[threadIdx.x >> 5] = ay;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    force[0] = (s_x[0] + s_x[1]) + (s_x[2] + s_x[3]);
    force[1] = (s_y[0] + s_y[1]) + (s_y[2] + s_y[3]);
  }
}

// Device address of g_noalloc_partials per device, as last looked up.  It is
// looked up again on every call made outside a stream capture (a cheap host
// call), so a context that was reset or replaced since is never served a
// stale address; inside a capture, where a first lookup could load the
// module, the address of the last call on that device is used.
std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace lbm

extern "C" lbm_status lbm_step_noalloc(const lbm_config* cfg, const float* src, float* dst,
                                       const uint8_t* kind, int64_t pitch, int64_t t,
                                       double* force) {
  using namespace lbm;
  auto bad = [](lbm_status st, const std::string& m) {
    set_last_error(m);
    return st;
  };
  if (!cfg || !src || !dst || !kind || !force)
    return bad(LBM_ERR_ARG, "cfg, src, dst, kind and force must be non-NULL");
  if (src == dst) return bad(LBM_ERR_ARG, "src and dst must be different buffers");
  if (cfg->precision != LBM_FP32)
    return bad(LBM_ERR_UNSUPPORTED, "lbm_step_noalloc supports FP32 populations only");
  if (cfg->nx < 1 || cfg->ny < 1) return bad(LBM_ERR_ARG, "nx and ny must be >= 1");
  if (!cfg->x_periodic && cfg->nx < 3) return bad(LBM_ERR_ARG, "open x needs nx >= 3");
  if (pitch < cfg->nx) return bad(LBM_ERR_ARG, "pitch must be >= nx");
  if ((int64_t)9 * cfg->ny * pitch >= ((int64_t)1 << 31))
    return bad(LBM_ERR_ARG, "9 * ny * pitch must stay below 2^31 elements");
  if (!(cfg->tau > 0.5) || !std::isfinite(cfg->tau)) return bad(LBM_ERR_ARG, "tau must be > 1/2");
  if (cfg->collision != LBM_BGK && cfg->collision != LBM_MRT)
    return bad(LBM_ERR_ARG, "unknown collision");
  if (!mrt_rates_valid(*cfg)) return bad(LBM_ERR_ARG, "MRT rates must lie in [0, 2)");
  if (!(std::fabs(cfg->u_in) < 1.0)) return bad(LBM_ERR_ARG, "|u_in| must be < 1");
  if (!(cfg->rho_out > 0.0)) return bad(LBM_ERR_ARG, "rho_out must be > 0");
  if (t < 0) return bad(LBM_ERR_ARG, "t must be >= 0");
  const int64_t tiles_x = ((int64_t)cfg->nx + 127) / 128;
  const int64_t strips = tiles_x * (((int64_t)cfg->ny + kRows - 1) / kRows);
  if (strips > kMaxStrips)
    return bad(LBM_ERR_ARG,
               "lattice too large for lbm_step_noalloc: it needs " + std::to_string(strips) +
                   " strips of 128 x 8 nodes but the static scratch holds " +
                   std::to_string(kMaxStrips) + " (e.g. 4096 x 2048 nodes at most)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bad(LBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return bad(LBM_ERR_UNSUPPORTED, "device index out of range");
  cudaStream_t st = (cudaStream_t)cfg->stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess)
    return bad(LBM_ERR_CUDA, std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e));
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
      if (e != cudaSuccess || !ptr)
        return bad(LBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_ptr[dev] = static_cast<double*>(ptr);
    } else if (!g_scratch_ptr[dev]) {
      return bad(LBM_ERR_STATE,
                 "the first lbm_step_noalloc call on a device must come before any stream "
                 "capture (it looks up the scratch array's device address)");
    }
    scratch = g_scratch_ptr[dev];
  }
  NoAllocParams p{};
  p.src = src;
  p.dst = dst;
  p.kind = kind;
  p.nx = cfg->nx;
  p.ny = cfg->ny;
  p.pitch = (int)pitch;
  p.plane = (int)(pitch * cfg->ny);
  p.omega = (float)(1.0 / cfg->tau);
  p.u_in = (float)cfg->u_in;
  p.rho_out = (float)cfg->rho_out;
  double rates[6];
  mrt_rates_of(*cfg, rates);
  p.mrt = {(float)rates[0], (float)rates[1], (float)rates[2],
           (float)rates[3], (float)rates[4], (float)rates[5]};
  p.v_amp = cfg->v_pert_amp;
  p.u_in_d = cfg->u_in;
  p.ramp_steps = cfg->ramp_steps;
  p.seed = cfg->seed;
  p.x_periodic = cfg->x_periodic;
  p.coll = cfg->collision;
  p.t = t;
  p.partials = scratch;
  p.force = force;
  noalloc_step_kernel<<<(unsigned)strips, 128, 0, st>>>(p);
  noalloc_reduce_kernel<<<1, 128, 0, st>>>(scratch, (int)strips, force);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bad(LBM_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return LBM_OK;
}
