// Fused stream-and-collide step of the D2Q9 lattice Boltzmann method and its
// helper kernels (geometry preparation, initialisation, export, mass).
//
// One launch advances every member lattice of a launch table by one time step
// (Sec. 2.1, Eq. 1, order of Fig. 1) in pull form: every node reads its nine
// incoming populations h_i(x - c_i) from its source buffer and writes its nine
// post-collision populations to the destination buffer, so each population is
// read once and written once per step (72 B per node in FP32).
//   - solid nodes (bit set in the solid mask): full-way bounce-back (Eq. 11)
//     stores the reversed incoming populations; counted links add their
//     momentum exchange (Eqs. 13-14) to an FP64 force accumulator;
//   - west column (open x): Zou & He velocity inlet, then collision;
//   - east column (open x): Zou & He pressure outflow (Eqs. 5-10) then
//     collision, or, with the NN or characteristic outflow, rebuilt by
//     boundary blocks of the same launch (Sec. 3.1, Eq. 15; Sec. 4, Eqs.
//     17-28) that run beside the stream-and-collide blocks (step_ext.cu);
//   - all other fluid nodes: BGK (Eq. 2) or MRT collision.
// The lattice is cut into strips of 128 columns x `rows` rows.  A launch table
// lists the member lattices (one simulation, or a batch of simulations of
// different sizes and parameters advanced together); each block handles one
// strip (or, for a single member, strides over its strips).  Each block writes
// an FP64 partial of its member's force; one extra block per member in the
// next launch (or a finalise launch) sums them in a fixed order into the
// member's force ring, so results are bitwise reproducible run to run.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lattice.cuh"
#include "sim.cuh"

#include "step_kernels.cuh"

namespace lbm {

__global__ void finalize_force_kernel(const StepParams p, int64_t tt) {
  reduce_force(p, blockIdx.x, tt);
  publish_reduced(p, blockIdx.x, tt);
}

__global__ void dataflow_reset_kernel(int64_t* strip_done, int n_strips, int64_t t,
                                      int64_t* reduced, int n_members, int64_t r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_strips) strip_done[i] = t;
  if (i < n_members) reduced[i] = r;
}

__global__ void set_t_kernel(int64_t* t_base, int64_t value) { *t_base = value; }

void launch_finalize_force(const StepParams& p, int64_t tt, cudaStream_t s) {
  finalize_force_kernel<<<p.n_members, 128, 0, s>>>(p, tt);
}

void launch_set_t(int64_t* t_base, int64_t value, cudaStream_t s) {
  set_t_kernel<<<1, 1, 0, s>>>(t_base, value);
}

void launch_dataflow_reset(int64_t* strip_done, int n_strips, int64_t t, int64_t* reduced,
                           int n_members, int64_t r, cudaStream_t s) {
  const int n = n_strips > n_members ? n_strips : n_members;
  dataflow_reset_kernel<<<(n + 255) / 256, 256, 0, s>>>(strip_done, n_strips, t, reduced,
                                                         n_members, r);
}

size_t step_bulk_smem(int prec, int stages) {
  // the ring (per-row stages; with FP16 storage the larger of those and the
  // row windows of variants 3, 4, 6), the full/empty barriers and the
  // alignment of the ring to 128 bytes
  int sb = prec == LBM_FP64 ? BulkLayout<double>::STAGE_BYTES
         : prec == LBM_FP32 ? BulkLayout<float>::STAGE_BYTES
                            : BulkLayout<__half>::STAGE_BYTES;
  if (prec == LBM_FP16DEV && WinLayout<__half>::SLOT_BYTES > sb) sb = WinLayout<__half>::SLOT_BYTES;
  return (size_t)stages * sb + (size_t)stages * 16 + 16 + 128;
}

// ---- variants and launch ------------------------------------------------------
int step_strips(int nx, int ny, int rows) {
  return ((nx + 127) / 128) * ((ny + rows - 1) / rows);
}

int step_ext_rows(int variant, int ext_kind, int prec) {
  // NN: kNnTcNodes nodes per block on the tensor cores (FP32 / FP16 storage),
  // kNnNodes with FP64; CBC: one node per thread but the first and last
  if (ext_kind == 1) return prec == LBM_FP64 ? kNnNodes : kNnTcNodes;
  return cbc_block_rows(step_variant_is_bulk(variant) ? kBulkThreads : 128);
}

int step_ext_blocks(int ny, int variant, int ext_kind, int prec) {
  const int per = step_ext_rows(variant, ext_kind, prec);
  return (ny + per - 1) / per;
}

bool step_variant_is_bulk(int variant) { return variant >= 3; }
bool step_variant_streams(int variant) { return variant == 4; }
bool step_variant_dynamic(int variant) { return variant == 5; }
bool step_variant_dataflow(int variant) { return variant == 6; }

int step_variants() { return kVariants; }


template <typename S, int COLL, int MINB, bool DYN>
static cudaError_t occ_bulk(int* per_sm) {
  const size_t smem = step_bulk_smem(prec_of<S>(), bulk_slots<S>());
  auto k = step_bulk_kernel<S, COLL, bulk_slots<S>(), MINB, false, DYN>;
  const cudaError_t e =
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, kBulkThreads, smem);
}

template <typename S, int COLL>
static cudaError_t occ(int variant, int* per_sm) {
  switch (variant) {
    case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 6, false>, 128, 0);
    case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 8, false>, 128, 0);
    case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, step_kernel<S, COLL, 10, false>, 128, 0);
    case 5: return occ_bulk<S, COLL, 6, true>(per_sm);
    default: return occ_bulk<S, COLL, 6, false>(per_sm);
  }
}

int step_max_blocks(int prec, int coll, int variant) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e;
  auto by_coll = [&](auto tag) {
    using S = decltype(tag);
    return coll == 0 ? occ<S, 0>(variant, &per_sm)
                     : (coll == 1 ? occ<S, 1>(variant, &per_sm) : occ<S, 2>(variant, &per_sm));
  };
  if (prec == LBM_FP64) e = by_coll(double{});
  else if (prec == LBM_FP32) e = by_coll(float{});
  else e = by_coll(__half{});
  if (e != cudaSuccess || sms <= 0 || per_sm <= 0) return 0;
  return sms * per_sm;
}

void launch_step(int prec, int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (p.nn_blocks > 0) {
    launch_step_ext(prec, coll, p, variant, blocks, s);   // step_ext.cu
    return;
  }
  if (prec == LBM_FP64) launch_c<double, false>(coll, p, variant, blocks, s);
  else if (prec == LBM_FP32) launch_c<float, false>(coll, p, variant, blocks, s);
  else launch_c<__half, false>(coll, p, variant, blocks, s);
}

// ---- geometry preparation --------------------------------------------------
// One thread per 32-cell word of a row: packs the solid bits and, for every
// counted solid node, the mask of links to fluid neighbours s - c_i.
__global__ void geometry_prep_kernel(const uint8_t* __restrict__ kind, int nx, int ny,
                                     int x_periodic, uint32_t* bits, int wpr,
                                     uint8_t* links, uint32_t* near_bits) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (w >= wpr || y >= ny) return;
  uint32_t word = 0, near = 0;
  for (int b = 0; b < 32; ++b) {
    const int x = w * 32 + b;
    if (x >= nx) break;
    const uint8_t k = kind[(int64_t)y * nx + x];
    if (k != LBM_CELL_FLUID) word |= 1u << b;
    // a counted solid node: links to the fluid nodes s - c_i; a fluid node:
    // links to the counted solid nodes x + c_i (the same links seen from the
    // fluid side, where the in-place step sums them)
    const uint8_t want = k == LBM_CELL_SOLID ? LBM_CELL_FLUID : LBM_CELL_SOLID;
    const int sgn = k == LBM_CELL_SOLID ? -1 : 1;
    uint8_t lk = 0;
    if (k == LBM_CELL_SOLID || k == LBM_CELL_FLUID) {
      for (int i = 1; i < 9; ++i) {
        int sx = x + sgn * cx(i);
        int sy = y + sgn * cy(i);
        sy = (sy + ny) % ny;
        if (sx < 0 || sx >= nx) {
          if (!x_periodic) continue;
          sx = (sx + nx) % nx;
        }
        if (kind[(int64_t)sy * nx + sx] == want) lk |= (uint8_t)(1u << (i - 1));
      }
    }
    links[(int64_t)y * nx + x] = lk;
    if (k == LBM_CELL_FLUID && lk) near |= 1u << b;
  }
  bits[(int64_t)y * wpr + w] = word;
  if (near_bits) near_bits[(int64_t)y * wpr + w] = near;
}

void launch_geometry_prep(const uint8_t* kind, int nx, int ny, int x_periodic, uint32_t* bits,
                          int words_per_row, uint8_t* links, uint32_t* near_bits, cudaStream_t s) {
  dim3 grid((words_per_row + 127) / 128, ny);
  geometry_prep_kernel<<<grid, 128, 0, s>>>(kind, nx, ny, x_periodic, bits, words_per_row, links,
                                            near_bits);
}

// ---- initialisation, import and export --------------------------------------
// Each works on rows [y0, y0 + rows) of the lattice; the dense host-side
// arrays (fields, or populations [9][rows][nx]) hold those rows only, so the
// host can stream a large lattice through a bounded scratch buffer.
template <typename S>
__global__ void init_eq_kernel(S* dst, int nx, int ny, int64_t pitch, int64_t plane,
                               const double* rho, const double* ux, const double* uy,
                               PopMap pm, int y0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y0 + (int)blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)blockIdx.y * nx + x;
  const double r = rho ? rho[c] : 1.0;
  const double u = ux ? ux[c] : 0.0;
  const double v = uy ? uy[c] : 0.0;
  double heq[9];
  heq_all<double>(r - 1.0, u, v, heq);
  for (int i = 0; i < 9; ++i) dst[pop_offset(pm, i, x, y, nx, ny, pitch, plane)] = from_r<S>(heq[i]);
}

void launch_init_equilibrium(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                             const double* rho, const double* ux, const double* uy,
                             cudaStream_t s, PopMap pm, int y0, int rows) {
  if (rows < 0) rows = ny - y0;
  if (rows <= 0) return;
  dim3 grid((nx + 127) / 128, rows);
  if (prec == LBM_FP64)
    init_eq_kernel<double><<<grid, 128, 0, s>>>((double*)dst, nx, ny, pitch, plane, rho, ux, uy,
                                                pm, y0);
  else if (prec == LBM_FP32)
    init_eq_kernel<float><<<grid, 128, 0, s>>>((float*)dst, nx, ny, pitch, plane, rho, ux, uy,
                                               pm, y0);
  else
    init_eq_kernel<__half><<<grid, 128, 0, s>>>((__half*)dst, nx, ny, pitch, plane, rho, ux, uy,
                                                pm, y0);
}

// f_i = h_i + w_i into a dense double[9][ny][nx]; moments into rho/ux/uy.
template <typename S>
__global__ void export_kernel(const S* src, int nx, int ny, int64_t pitch, int64_t plane,
                              double* f_out, double* rho, double* ux, double* uy, PopMap pm,
                              int y0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y0 + (int)blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)blockIdx.y * nx + x;
  const int64_t n = (int64_t)nx * gridDim.y;
  double f[9];
  for (int i = 0; i < 9; ++i) {
    f[i] = (double)to_r<double>(src[pop_offset(pm, i, x, y, nx, ny, pitch, plane)]) +
           wgt<double>(i);
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
                   double* f_out, double* rho, double* ux, double* uy, cudaStream_t s,
                   PopMap pm, int y0, int rows) {
  if (rows < 0) rows = ny - y0;
  if (rows <= 0) return;
  dim3 grid((nx + 127) / 128, rows);
  if (prec == LBM_FP64)
    export_kernel<double><<<grid, 128, 0, s>>>((const double*)src, nx, ny, pitch, plane, f_out,
                                               rho, ux, uy, pm, y0);
  else if (prec == LBM_FP32)
    export_kernel<float><<<grid, 128, 0, s>>>((const float*)src, nx, ny, pitch, plane, f_out, rho,
                                              ux, uy, pm, y0);
  else
    export_kernel<__half><<<grid, 128, 0, s>>>((const __half*)src, nx, ny, pitch, plane, f_out,
                                               rho, ux, uy, pm, y0);
}

template <typename S>
__global__ void import_kernel(S* dst, int nx, int ny, int64_t pitch, int64_t plane,
                              const double* f_in, PopMap pm, int y0) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = y0 + (int)blockIdx.y;
  if (x >= nx) return;
  const int64_t c = (int64_t)blockIdx.y * nx + x;
  const int64_t n = (int64_t)nx * gridDim.y;
  for (int i = 0; i < 9; ++i)
    dst[pop_offset(pm, i, x, y, nx, ny, pitch, plane)] = from_r<S>(f_in[i * n + c] - wgt<double>(i));
}

void launch_import(int prec, void* dst, int nx, int ny, int64_t pitch, int64_t plane,
                   const double* f_in, cudaStream_t s, PopMap pm, int y0, int rows) {
  if (rows < 0) rows = ny - y0;
  if (rows <= 0) return;
  dim3 grid((nx + 127) / 128, rows);
  if (prec == LBM_FP64)
    import_kernel<double><<<grid, 128, 0, s>>>((double*)dst, nx, ny, pitch, plane, f_in, pm, y0);
  else if (prec == LBM_FP32)
    import_kernel<float><<<grid, 128, 0, s>>>((float*)dst, nx, ny, pitch, plane, f_in, pm, y0);
  else
    import_kernel<__half><<<grid, 128, 0, s>>>((__half*)dst, nx, ny, pitch, plane, f_in, pm, y0);
}

// ---- total mass: per-row partial sums, then one block sums the rows --------
template <typename S>
__global__ void mass_rows_kernel(const S* src, int nx, int ny, int64_t pitch, int64_t plane,
                                 double* partials, PopMap pm) {
  const int y = blockIdx.x;
  double acc = 0.0;
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double cell = 1.0;   // sum of the weights
    for (int i = 0; i < 9; ++i)
      cell += (double)to_r<double>(src[pop_offset(pm, i, x, y, nx, ny, pitch, plane)]);
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
                 double* partials, int n_partials, double* out, cudaStream_t s, PopMap pm) {
  (void)n_partials;
  if (prec == LBM_FP64)
    mass_rows_kernel<double><<<ny, 256, 0, s>>>((const double*)src, nx, ny, pitch, plane, partials,
                                                pm);
  else if (prec == LBM_FP32)
    mass_rows_kernel<float><<<ny, 256, 0, s>>>((const float*)src, nx, ny, pitch, plane, partials,
                                               pm);
  else
    mass_rows_kernel<__half><<<ny, 256, 0, s>>>((const __half*)src, nx, ny, pitch, plane, partials,
                                                pm);
  sum_partials_kernel<<<1, 1024, 0, s>>>(partials, ny, out);
}

}  // namespace lbm
