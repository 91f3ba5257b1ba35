// Fused stream-and-collide step of the D2Q9 lattice Boltzmann method and its
// helper kernels (geometry preparation, initialisation, export, mass).
//
// One launch advances the whole lattice by one time step (Sec. 2.1, Eq. 1,
// order of Fig. 1) in pull form: every node reads its nine incoming
// populations h_i(x - c_i) from the source buffer and writes its nine
// post-collision populations to the destination buffer, so each population is
// read once and written once per step (72 B per node in FP32).
//   - solid nodes (bit set in the solid mask): full-way bounce-back (Eq. 11)
//     stores the reversed incoming populations; counted links add their
//     momentum exchange (Eqs. 13-14) to an FP64 force accumulator;
//   - west column (open x): Zou & He velocity inlet, then collision;
//   - east column (open x): Zou & He pressure outflow (Eqs. 5-10) then
//     collision, or left to the outflow kernel (NN, CBC);
//   - all other fluid nodes: BGK (Eq. 2) or MRT collision.
// Each block writes an FP64 partial of the force; an extra block of the next
// launch (or a one-block finalise kernel) sums the partials in a fixed order
// into the force ring, so results are bitwise reproducible run to run.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "sim.cuh"

namespace lbm {

template <typename S>
__device__ __forceinline__ S ldg(const S* p) { return __ldg(p); }

template <typename R>
__device__ __forceinline__ void warp_sum2(R& a, R& b) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, off);
    b += __shfl_down_sync(0xffffffffu, b, off);
  }
}

// Pull-load the nine incoming populations of node (x, y): h_i = A_i(x - c_i).
// Offsets are 32-bit: the library keeps 9 * plane below 2^31 elements.
template <typename S, typename R>
__device__ __forceinline__ void pull_row(const S* __restrict__ A, int plane, int rc, int rm,
                                         int rp, int x, int xm, int xp, R h[9]) {
  h[0] = to_r<R>(ldg(A + rc + x));
  h[1] = to_r<R>(ldg(A + 1 * plane + rc + xm));
  h[2] = to_r<R>(ldg(A + 2 * plane + rm + x));
  h[3] = to_r<R>(ldg(A + 3 * plane + rc + xp));
  h[4] = to_r<R>(ldg(A + 4 * plane + rp + x));
  h[5] = to_r<R>(ldg(A + 5 * plane + rm + xm));
  h[6] = to_r<R>(ldg(A + 6 * plane + rm + xp));
  h[7] = to_r<R>(ldg(A + 7 * plane + rp + xp));
  h[8] = to_r<R>(ldg(A + 8 * plane + rp + xm));
}

template <typename R>
__device__ __forceinline__ bool nonfinite(R v) { return !(fabs(v) < R(1e30)); }

template <typename R> struct Scalars;
template <> struct Scalars<float> {
  float omega, u_in, rho_out;
  MrtRates<float> mrt;
  __device__ explicit Scalars(const StepParams& p)
      : omega(p.omega_f), u_in(p.u_in_f), rho_out(p.rho_out_f),
        mrt{p.mrt_f[0], p.mrt_f[1], p.mrt_f[2], p.mrt_f[3]} {}
};
template <> struct Scalars<double> {
  double omega, u_in, rho_out;
  MrtRates<double> mrt;
  __device__ explicit Scalars(const StepParams& p)
      : omega(p.omega), u_in(p.u_in), rho_out(p.rho_out),
        mrt{p.mrt_se, p.mrt_seps, p.mrt_sq, p.mrt_snu} {}
};

// Fixed-order sum of the block partials of step tt into the force ring
// (executed by one block of 128 threads).
__device__ void reduce_force(const StepParams& p, int64_t tt, int nb) {
  __shared__ double s_x[4], s_y[4];
  const double* part = p.partials + (size_t)(tt & 1) * 2 * p.partial_stride;
  double ax = 0.0, ay = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    ax += part[2 * b];
    ay += part[2 * b + 1];
  }
  warp_sum2(ax, ay);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_x[warp] = ax; s_y[warp] = ay; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t k = tt % p.ring_cap;
    p.ring[2 * k] = (s_x[0] + s_x[1]) + (s_x[2] + s_x[3]);
    p.ring[2 * k + 1] = (s_y[0] + s_y[1]) + (s_y[2] + s_y[3]);
  }
}

// One block = 128 consecutive x of a strip of `rows` rows; blocks stride over
// the strips (grid sized to the resident capacity by the host).  Each thread
// walks its column down the strip and prefetches the next row's populations
// and solid-mask word while the current row collides.  The extra last block
// does no lattice work: it sums the previous step's force partials, so no
// block waits at the end of a step.
template <typename S, int COLL, int MINB>
__global__ void __launch_bounds__(128, MINB) step_kernel(const StepParams p) {
  using R = typename Compute<S>::R;
  const int nblocks = gridDim.x - 1;
  const int64_t t = p.t_base ? *p.t_base + p.t_offset : p.t;
  if ((int)blockIdx.x == nblocks) {
    if (p.reduce_prev && t >= 1) reduce_force(p, t - 1, p.prev_blocks);
    return;
  }
  const S* __restrict__ A = static_cast<const S*>(p.src);
  S* __restrict__ B = static_cast<S*>(p.dst);
  const int plane = (int)p.plane, pitch = (int)p.pitch;
  const int nx = p.nx, ny = p.ny, rows = p.rows;
  const int tiles_x = (nx + 127) >> 7;
  const int strips = tiles_x * ((ny + rows - 1) / rows);
  const Scalars<R> sc(p);

  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;

  for (int s = blockIdx.x; s < strips; s += nblocks) {
    const int tx = s % tiles_x;
    const int y0 = (s / tiles_x) * rows;
    const int y1 = min(y0 + rows, ny);
    const int x = (tx << 7) + threadIdx.x;
    if (x >= nx) continue;
    const bool west = !p.x_periodic && x == 0;
    const bool east = !p.x_periodic && x == nx - 1;
    if (east && p.east_mode == EAST_EXTERNAL) continue;
    const int xm = x == 0 ? nx - 1 : x - 1;
    const int xp = x == nx - 1 ? 0 : x + 1;
    const uint32_t* bits = p.solid_bits + (x >> 5);
    const uint32_t bit = 1u << (x & 31);

    R h[9];
    uint32_t word;
    {
      const int ym = y0 == 0 ? ny - 1 : y0 - 1;
      const int yp = y0 + 1 == ny ? 0 : y0 + 1;
      pull_row<S, R>(A, plane, y0 * pitch, ym * pitch, yp * pitch, x, xm, xp, h);
      word = __ldg(bits + y0 * p.words_per_row);
    }
    for (int y = y0; y < y1; ++y) {
      R hn[9];
      uint32_t word_n = 0;
      const bool more = y + 1 < y1;
      if (more) {
        const int y2 = y + 1;
        const int yp = y2 + 1 == ny ? 0 : y2 + 1;
        pull_row<S, R>(A, plane, y2 * pitch, y * pitch, yp * pitch, x, xm, xp, hn);
        word_n = __ldg(bits + y2 * p.words_per_row);
      }
      const int o = y * pitch + x;
      if (word & bit) {
        // solid: momentum exchange over counted links, then full-way bounce-back
        const unsigned lk = __ldg(p.links + (int64_t)y * nx + x);
        if (lk) {
          touched = true;
#pragma unroll
          for (int i = 1; i < 9; ++i) {
            if ((lk >> (i - 1)) & 1u) {
              // f_i arriving now + f_ibar that bounce-back stored here last step
              const double v = (double)h[i] + (double)to_r<R>(ldg(A + opp(i) * plane + o)) +
                               2.0 * wgt<double>(i);
              fx += cx(i) * v;
              fy += cy(i) * v;
            }
          }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) B[i * plane + o] = from_r<S>(h[opp(i)]);
      } else {
        if (west) {
          const R v = (R)inlet_perturbation(p.seed, t, y, p.v_amp);
          zouhe_west<R>(h, sc.u_in, v);
        } else if (east) {
          zouhe_east<R>(h, sc.rho_out);
        }
        R drho, ux, uy;
        if (COLL == 0)
          collide_bgk<R>(h, sc.omega, drho, ux, uy);
        else
          collide_mrt<R>(h, sc.mrt, drho, ux, uy);
        bad |= nonfinite(drho);
#pragma unroll
        for (int i = 0; i < 9; ++i) B[i * plane + o] = from_r<S>(h[i]);
      }
      if (more) {
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = hn[i];
        word = word_n;
      }
    }
  }

  if (bad) atomicOr(p.status, DEV_NONFINITE);

  // ---- block partial of the force (FP64 work only where links were hit) ---
  double* part = p.partials + (size_t)(t & 1) * 2 * p.partial_stride;
  if (!__syncthreads_or(touched)) {
    if (threadIdx.x == 0) {
      part[2 * blockIdx.x] = 0.0;
      part[2 * blockIdx.x + 1] = 0.0;
    }
    return;
  }
  __shared__ double s_fx[4], s_fy[4];
  warp_sum2(fx, fy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_fx[warp] = fx; s_fy[warp] = fy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = (s_fx[0] + s_fx[1]) + (s_fx[2] + s_fx[3]);
    part[2 * blockIdx.x + 1] = (s_fy[0] + s_fy[1]) + (s_fy[2] + s_fy[3]);
  }
}

__global__ void finalize_force_kernel(const StepParams p, int64_t tt, int nb) {
  reduce_force(p, tt, nb);
}

__global__ void set_t_kernel(int64_t* t_base, int64_t value) { *t_base = value; }

void launch_finalize_force(const StepParams& p, int64_t tt, int blocks, cudaStream_t s) {
  finalize_force_kernel<<<1, 128, 0, s>>>(p, tt, blocks);
}

void launch_set_t(int64_t* t_base, int64_t value, cudaStream_t s) {
  set_t_kernel<<<1, 1, 0, s>>>(t_base, value);
}

int step_blocks(int nx, int ny, int rows, int max_blocks) {
  const int tiles_x = (nx + 127) / 128;
  const int strips = tiles_x * ((ny + rows - 1) / rows);
  return strips < max_blocks ? strips : max_blocks;
}

// Register-budget variants of the step kernel: __launch_bounds__ minimum
// resident blocks of 128 threads per SM (more blocks = fewer registers).
constexpr int kVariants = 3;
constexpr int kMinBlocks[kVariants] = {6, 8, 10};

template <typename S, int COLL>
static cudaError_t occ(int variant, int* per_sm) {
  switch (variant) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 6>, 128, 0);
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 8>, 128, 0);
    default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 10>, 128, 0);
  }
}

int step_variants() { return kVariants; }

int step_max_blocks(int prec, int coll, int variant) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  if (prec == LBM_FP64)
    e = coll == LBM_BGK ? occ<double, 0>(variant, &per_sm) : occ<double, 1>(variant, &per_sm);
  else if (prec == LBM_FP32)
    e = coll == LBM_BGK ? occ<float, 0>(variant, &per_sm) : occ<float, 1>(variant, &per_sm);
  else
    e = coll == LBM_BGK ? occ<__half, 0>(variant, &per_sm) : occ<__half, 1>(variant, &per_sm);
  if (e != cudaSuccess || sms <= 0 || per_sm <= 0) return 0;
  return sms * per_sm;
}

template <typename S, int COLL>
static void launch_v(const StepParams& p, int variant, int blocks, cudaStream_t s) {
  switch (variant) {
    case 0: step_kernel<S, COLL, 6><<<blocks + 1, 128, 0, s>>>(p); break;
    case 1: step_kernel<S, COLL, 8><<<blocks + 1, 128, 0, s>>>(p); break;
    default: step_kernel<S, COLL, 10><<<blocks + 1, 128, 0, s>>>(p); break;
  }
}

void launch_step(int prec, int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (prec == LBM_FP64) {
    if (coll == LBM_BGK) launch_v<double, 0>(p, variant, blocks, s);
    else launch_v<double, 1>(p, variant, blocks, s);
  } else if (prec == LBM_FP32) {
    if (coll == LBM_BGK) launch_v<float, 0>(p, variant, blocks, s);
    else launch_v<float, 1>(p, variant, blocks, s);
  } else {
    if (coll == LBM_BGK) launch_v<__half, 0>(p, variant, blocks, s);
    else launch_v<__half, 1>(p, variant, blocks, s);
  }
}

// ---- geometry preparation --------------------------------------------------
// One thread per 32-cell word of a row: packs the solid bits and, for every
// counted solid node, the mask of links to fluid neighbours s - c_i.
__global__ void geometry_prep_kernel(const uint8_t* __restrict__ kind, int nx, int ny,
                                     int x_periodic, uint32_t* bits, int wpr,
                                     uint8_t* links) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (w >= wpr || y >= ny) return;
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const int x = w * 32 + b;
    if (x >= nx) break;
    const uint8_t k = kind[(int64_t)y * nx + x];
    if (k != LBM_CELL_FLUID) word |= 1u << b;
    uint8_t lk = 0;
    if (k == LBM_CELL_SOLID) {
      for (int i = 1; i < 9; ++i) {
        int sx = x - cx(i);
        int sy = y - cy(i);
        sy = (sy + ny) % ny;
        if (sx < 0 || sx >= nx) {
          if (!x_periodic) continue;
          sx = (sx + nx) % nx;
        }
        if (kind[(int64_t)sy * nx + sx] == LBM_CELL_FLUID) lk |= (uint8_t)(1u << (i - 1));
      }
    }
    links[(int64_t)y * nx + x] = lk;
  }
  bits[(int64_t)y * wpr + w] = word;
}

void launch_geometry_prep(const uint8_t* kind, int nx, int ny, int x_periodic, uint32_t* bits,
                          int words_per_row, uint8_t* links, cudaStream_t s) {
  dim3 grid((words_per_row + 127) / 128, ny);
  geometry_prep_kernel<<<grid, 128, 0, s>>>(kind, nx, ny, x_periodic, bits, words_per_row, links);
}

// ---- initialisation, import and export --------------------------------------
template <typename S>
__global__ void init_eq_kernel(S* dst, int nx, int ny, int64_t pitch, int64_t plane,
                               const double* rho, const double* ux, const double* uy) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)y * nx + x;
  const double r = rho ? rho[c] : 1.0;
  const double u = ux ? ux[c] : 0.0;
  const double v = uy ? uy[c] : 0.0;
  double heq[9];
  heq_all<double>(r - 1.0, u, v, heq);
  for (int i = 0; i < 9; ++i) dst[i * plane + (int64_t)y * pitch + x] = from_r<S>(heq[i]);
}

void launch_init_equilibrium(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                             const double* rho, const double* ux, const double* uy,
                             cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny);
  if (prec == LBM_FP64)
    init_eq_kernel<double><<<grid, 128, 0, s>>>((double*)dst, nx, ny, pitch, plane, rho, ux, uy);
  else if (prec == LBM_FP32)
    init_eq_kernel<float><<<grid, 128, 0, s>>>((float*)dst, nx, ny, pitch, plane, rho, ux, uy);
  else
    init_eq_kernel<__half><<<grid, 128, 0, s>>>((__half*)dst, nx, ny, pitch, plane, rho, ux, uy);
}

// f_i = h_i + w_i into a dense double[9][ny][nx]; moments into rho/ux/uy.
template <typename S>
__global__ void export_kernel(const S* src, int nx, int ny, int64_t pitch, int64_t plane,
                              double* f_out, double* rho, double* ux, double* uy) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)y * nx + x;
  const int64_t n = (int64_t)nx * ny;
  double f[9];
  for (int i = 0; i < 9; ++i) {
    f[i] = (double)to_r<double>(src[i * plane + (int64_t)y * pitch + x]) + wgt<double>(i);
    if (f_out) f_out[i * n + c] = f[i];
  }
  double r = 0.0, jx = 0.0, jy = 0.0;
  for (int i = 0; i < 9; ++i) {
    r += f[i];
    jx += cx(i) * f[i];
    jy += cy(i) * f[i];
  }
  if (rho) rho[c] = r;
  if (ux) ux[c] = jx / r;
  if (uy) uy[c] = jy / r;
}

void launch_export(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                   double* f_out, double* rho, double* ux, double* uy, cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny);
  if (prec == LBM_FP64)
    export_kernel<double><<<grid, 128, 0, s>>>((const double*)src, nx, ny, pitch, plane, f_out,
                                               rho, ux, uy);
  else if (prec == LBM_FP32)
    export_kernel<float><<<grid, 128, 0, s>>>((const float*)src, nx, ny, pitch, plane, f_out, rho,
                                              ux, uy);
  else
    export_kernel<__half><<<grid, 128, 0, s>>>((const __half*)src, nx, ny, pitch, plane, f_out,
                                               rho, ux, uy);
}

template <typename S>
__global__ void import_kernel(S* dst, int nx, int ny, int64_t pitch, int64_t plane,
                              const double* f_in) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)y * nx + x;
  const int64_t n = (int64_t)nx * ny;
  for (int i = 0; i < 9; ++i)
    dst[i * plane + (int64_t)y * pitch + x] = from_r<S>(f_in[i * n + c] - wgt<double>(i));
}

void launch_import(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                   const double* f_in, cudaStream_t s) {
  dim3 grid((nx + 127) / 128, ny);
  if (prec == LBM_FP64)
    import_kernel<double><<<grid, 128, 0, s>>>((double*)dst, nx, ny, pitch, plane, f_in);
  else if (prec == LBM_FP32)
    import_kernel<float><<<grid, 128, 0, s>>>((float*)dst, nx, ny, pitch, plane, f_in);
  else
    import_kernel<__half><<<grid, 128, 0, s>>>((__half*)dst, nx, ny, pitch, plane, f_in);
}

// ---- total mass: per-row partial sums, then one block sums the rows --------
template <typename S>
__global__ void mass_rows_kernel(const S* src, int nx, int ny, int64_t pitch, int64_t plane,
                                 double* partials) {
  const int y = blockIdx.x;
  double acc = 0.0;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double cell = 1.0;   // sum of the weights
    for (int i = 0; i < 9; ++i) cell += (double)to_r<double>(src[i * plane + (int64_t)y * pitch + x]);
    acc += cell;
  }
  __shared__ double sh[32];
  double dummy = 0.0;
  warp_sum2(acc, dummy);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    partials[y] = s;
  }
}

__global__ void sum_partials_kernel(const double* partials, int n, double* out) {
  double acc = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) acc += partials[k];
  __shared__ double sh[32];
  double dummy = 0.0;
  warp_sum2(acc, dummy);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    *out = s;
  }
}

void launch_mass(int prec, const void* src, int nx, int ny, int64_t pitch, int64_t plane,
                 double* partials, int n_partials, double* out, cudaStream_t s) {
  (void)n_partials;
  if (prec == LBM_FP64)
    mass_rows_kernel<double><<<ny, 256, 0, s>>>((const double*)src, nx, ny, pitch, plane, partials);
  else if (prec == LBM_FP32)
    mass_rows_kernel<float><<<ny, 256, 0, s>>>((const float*)src, nx, ny, pitch, plane, partials);
  else
    mass_rows_kernel<__half><<<ny, 256, 0, s>>>((const __half*)src, nx, ny, pitch, plane, partials);
  sum_partials_kernel<<<1, 1024, 0, s>>>(partials, ny, out);
}

}  // namespace lbm
