// Kernel templates of the fused step (included by step.cu and step_nn.cu).
//
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
//     collision, or, with the NN outflow, rebuilt by network blocks of the same
//     launch (Sec. 3.1, Eq. 15) that run beside the stream-and-collide blocks;
//   - all other fluid nodes: BGK (Eq. 2) or MRT collision.
// The lattice is cut into strips of 128 columns x `rows` rows.  A launch table
// lists the member lattices (one simulation, or a batch of simulations of
// different sizes and parameters advanced together); each block handles one
// strip (or, for a single member, strides over its strips).  Each block writes
// an FP64 partial of its member's force; one extra block per member in the
// next launch (or a finalise launch) sums them in a fixed order into the
// member's force ring, so results are bitwise reproducible run to run.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include "lattice.cuh"
#include "mma_tf32.cuh"
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

// hidden-layer activation of the outflow network: 0 tanh, 1 LeakyReLU (0.01)
template <typename R>
__device__ __forceinline__ R act_hidden(R a, int act) {
  if (act == 0) return tanh(a);
  return a > R(0) ? a : R(0.01) * a;
}

// A member's scalars in the compute precision (FP32 copies are made on the
// host: GB300's FP64 pipe is narrow).  The MRT rates are not among them: they
// are read from the member record where the collision needs them (mrt_of), so
// a strip loop does not hold six more registers.
template <typename R> struct Scalars;
template <> struct Scalars<float> {
  float omega, u_in, rho_out;
  __device__ explicit Scalars(const Member& m)
      : omega(m.omega_f), u_in(m.u_in_f), rho_out(m.rho_out_f) {}
};
template <> struct Scalars<double> {
  double omega, u_in, rho_out;
  __device__ explicit Scalars(const Member& m)
      : omega(m.omega), u_in(m.u_in), rho_out(m.rho_out) {}
};

template <typename R> __device__ __forceinline__ MrtRates<R> mrt_of(const Member& m);
template <> __device__ __forceinline__ MrtRates<float> mrt_of<float>(const Member& m) {
  return {m.mrt_f[0], m.mrt_f[1], m.mrt_f[2], m.mrt_f[3], m.mrt_f[4], m.mrt_f[5]};
}
template <> __device__ __forceinline__ MrtRates<double> mrt_of<double>(const Member& m) {
  return {m.mrt[0], m.mrt[1], m.mrt[2], m.mrt[3], m.mrt[4], m.mrt[5]};
}

// Programmatic dependent launch: a step kernel lets the next one be
// scheduled early (it then does its set-up while this one drains) and waits
// for the previous step's grid to complete before it touches populations.
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int64_t step_index(const StepParams& p) {
  return p.t_base ? *p.t_base + p.t_offset : p.t;
}

// ---- dataflow between consecutive step launches (variant 6) ------------------
// A strip's step t reads the populations that step t-1 wrote in the 3 x 3
// strips around it (pull halo of one node, both axes periodic at worst) and
// overwrites the buffer that those strips read in step t-1.  So instead of
// waiting for the whole previous launch (griddepcontrol.wait) a block waits
// until those nine strips have completed step t-1, and the next launch's
// blocks fill the SMs while this one drains.  Every block of a launch starts
// before any block of the next one does (a dependent launch begins once all
// blocks of its predecessor have triggered it, which they do on entry), so a
// block only ever waits for blocks that are already running.  Flags count
// completed steps and are published with release/acquire at GPU scope; waits
// are bounded in time and latch DEV_TIMEOUT when they give up.
__device__ __forceinline__ int64_t ld_acquire(const int64_t* ptr) {
  int64_t v;
  asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(ptr) : "memory");
  return v;
}
__device__ __forceinline__ int64_t ld_relaxed(const int64_t* ptr) {
  int64_t v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(ptr) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int64_t* ptr, int64_t v) {
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(ptr), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t v;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
  return v;
}

constexpr uint64_t kFlagWaitNs = 2000000000ull;   // a flag wait gives up after 2 s

// A wait that has not been satisfied at once also gives up as soon as its
// member's status word holds DEV_TIMEOUT: once one wait of a launch has run
// out, the flags it depends on cannot all arrive, and every further block
// would otherwise spend its own 2 s before the host can see the fault.
__device__ __forceinline__ bool timed_out_already(const int* status) {
  return (*reinterpret_cast<const volatile int*>(status) & DEV_TIMEOUT) != 0;
}

// Bounded wait until *ptr >= v; false if it gave up.
__device__ inline bool wait_at_least(const int64_t* ptr, int64_t v, const int* status) {
  if (ld_acquire(ptr) >= v) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t k = 0; k < (1u << 24); ++k) {
    __nanosleep(200);
    if (ld_acquire(ptr) >= v) return true;
    if (global_ns() - t0 > kFlagWaitNs || timed_out_already(status)) return false;
  }
  return false;
}

// Local strip ls of member m: wait until its 3 x 3 neighbourhood (periodic
// in both axes: the edge columns read the opposite edge) has completed t steps.
// The nine flags are read with relaxed loads issued together (one round trip
// instead of nine serialised acquires); the fence after the last poll makes
// the whole wait an acquire of every flag it saw.
__device__ inline bool wait_strip_neighbours(const StepParams& p, const Member& m, int ls,
                                             int64_t t) {
  const int tiles = m.tiles_x;
  const int nrow = (m.ny + p.rows - 1) / p.rows;
  const int r0 = ls / tiles, c0 = ls % tiles;
  const int64_t* f[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    const int r = (r0 + j / 3 - 1 + nrow) % nrow;
    const int c = (c0 + j % 3 - 1 + tiles) % tiles;
    f[j] = p.strip_done + m.strip_first + r * tiles + c;
  }
  uint64_t t0 = 0;
  for (uint32_t k = 0; k < (1u << 24); ++k) {
    int64_t v[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) v[j] = ld_relaxed(f[j]);
    bool all = true;
#pragma unroll
    for (int j = 0; j < 9; ++j) all &= v[j] >= t;
    if (all) {
      __threadfence();
      return true;
    }
    if (k == 0) t0 = global_ns();
    else if (global_ns() - t0 > kFlagWaitNs || timed_out_already(m.status)) break;
    __nanosleep(200);
  }
  __threadfence();
  return false;
}

// after a reduction of member k's forces through step index tt
__device__ __forceinline__ void publish_reduced(const StepParams& p, int k, int64_t tt) {
  if (p.reduced && threadIdx.x == 0) {
    __threadfence();
    st_release(p.reduced + k, tt + 1);
  }
}

// Fixed-order sum of member k's block partials of step tt into its force ring
// (one block of 128 threads).
__device__ inline void reduce_force(const StepParams& p, int k, int64_t tt) {
  __shared__ double s_x[8], s_y[8];
  const Member& m = p.members[k];
  const double* part = p.partials + (size_t)(tt & 1) * 2 * p.partial_stride;
  double ax = 0.0, ay = 0.0;
  for (int b = m.part_first + threadIdx.x; b < m.part_first + m.part_count; b += blockDim.x) {
    ax += part[2 * b];
    ay += part[2 * b + 1];
  }
  warp_sum2(ax, ay);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_x[warp] = ax; s_y[warp] = ay; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bx = 0.0, by = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { bx += s_x[w]; by += s_y[w]; }
    const int64_t slot = tt % m.ring_cap;
    m.ring[2 * slot] = bx;
    m.ring[2 * slot + 1] = by;
  }
}

// Solid node: momentum exchange over counted links (FP64), then full-way
// bounce-back store.  Shared by both kernel families.
template <typename S, typename R>
__device__ __forceinline__ void solid_node(const S* __restrict__ A, S* __restrict__ B,
                                           const Member& m, int x, int y, int o, const R h[9],
                                           double& fx, double& fy, bool& touched) {
  const unsigned lk = __ldg(m.links + (int64_t)y * m.nx + x);
  if (lk) {
    touched = true;
    // this node's links summed in the compute precision (at most 8 terms of
    // similar size), then accumulated in FP64 across nodes, rows and blocks
    R sx = R(0), sy = R(0);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
      if ((lk >> (i - 1)) & 1u) {
        // f_i arriving now + f_ibar that bounce-back stored here last step
        const R v = h[i] + to_r<R>(__ldcg(A + opp(i) * m.plane + o)) + R(2) * wgt<R>(i);
        sx += R(cx(i)) * v;
        sy += R(cy(i)) * v;
      }
    }
    fx += (double)sx;
    fy += (double)sy;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[opp(i)]);
}

// Fluid node: open boundaries, collision, store.
template <typename S, typename R, int COLL>
__device__ __forceinline__ void fluid_node(S* __restrict__ B, const Member& m,
                                           const Scalars<R>& sc, int64_t t, bool west,
                                           bool east, int y, int o, R h[9], bool& bad) {
  if (west) {
    const R v = m.v_amp != 0.0 ? (R)inlet_perturbation(m.seed, t, y, m.v_amp) : R(0);
    const R u = m.ramp_steps > 0 ? (R)inlet_velocity(m.u_in, m.ramp_steps, t) : sc.u_in;
    zouhe_west<R>(h, u, v);
  } else if (east) {
    zouhe_east<R>(h, sc.rho_out);
  }
  R drho, ux, uy;
  // COLL 0: BGK, 1: MRT, 2: the member's own choice (mixed batches)
  if (COLL == 0 || (COLL == 2 && m.coll == LBM_BGK))
    collide_bgk<R>(h, sc.omega, drho, ux, uy);
  else
    collide_mrt<R>(h, mrt_of<R>(m), drho, ux, uy);
  bad |= nonfinite(drho);
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[i]);
}

// Block partial of the force (FP64 shuffles only where a counted link was hit)
// and one block-wide vote on non-finite densities.
__device__ __forceinline__ void write_partial(const StepParams& p, int64_t t, int slot, double fx,
                                              double fy, bool touched, bool bad, int* status) {
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, DEV_NONFINITE);
  if (slot < 0) return;   // a strip without counted solid nodes has no partial
  double* part = p.partials + (size_t)(t & 1) * 2 * p.partial_stride;
  if (!__syncthreads_or(touched)) {
    if (threadIdx.x == 0) {
      part[2 * slot] = 0.0;
      part[2 * slot + 1] = 0.0;
    }
    return;
  }
  __shared__ double s_fx[8], s_fy[8];
  warp_sum2(fx, fy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_fx[warp] = fx; s_fy[warp] = fy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bx = 0.0, by = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { bx += s_fx[w]; by += s_fy[w]; }
    part[2 * slot] = bx;
    part[2 * slot + 1] = by;
  }
}

// ---- register-pipelined kernel ---------------------------------------------
// Each thread walks its column down a strip and prefetches the next row's
// populations and solid-mask word while the current row collides.  With one
// member (p.persistent) blocks stride over its strips on a grid sized to the
// resident capacity; otherwise each block handles exactly one strip of the
// member given by the strip table.
template <typename S, int COLL>
__device__ __forceinline__ void reg_strip(const StepParams& p, const Member& m,
                                          const Scalars<typename Compute<S>::R>& sc, int64_t t,
                                          int s, double& fx, double& fy, bool& touched,
                                          bool& bad) {
  using R = typename Compute<S>::R;
  const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  const int plane = m.plane, pitch = m.pitch, nx = m.nx, ny = m.ny;
  const int tx = s % m.tiles_x;
  const int y0 = (s / m.tiles_x) * p.rows;
  const int y1 = min(y0 + p.rows, ny);
  const int x = (tx << 7) + threadIdx.x;
  if (x >= nx) return;
  const bool west = !m.x_periodic && x == 0;
  const bool east = !m.x_periodic && x == nx - 1;
  // the network blocks rebuild external east fluid nodes; solid ones stay here
  const bool ext = east && m.east_mode == EAST_EXTERNAL;
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x == nx - 1 ? 0 : x + 1;
  const uint32_t* bits = m.solid_bits + (x >> 5);
  const uint32_t bit = 1u << (x & 31);

  R h[9];
  uint32_t word;
  {
    const int ym = y0 == 0 ? ny - 1 : y0 - 1;
    const int yp = y0 + 1 == ny ? 0 : y0 + 1;
    pull_row<S, R>(A, plane, y0 * pitch, ym * pitch, yp * pitch, x, xm, xp, h);
    word = __ldg(bits + y0 * m.words_per_row);
  }
  for (int y = y0; y < y1; ++y) {
    R hn[9];
    uint32_t word_n = 0;
    const bool more = y + 1 < y1;
    if (more) {
      const int y2 = y + 1;
      const int yp = y2 + 1 == ny ? 0 : y2 + 1;
      pull_row<S, R>(A, plane, y2 * pitch, y * pitch, yp * pitch, x, xm, xp, hn);
      word_n = __ldg(bits + y2 * m.words_per_row);
    }
    const int o = y * pitch + x;
    if (word & bit)
      solid_node<S, R>(A, B, m, x, y, o, h, fx, fy, touched);
    else if (!ext)
      fluid_node<S, R, COLL>(B, m, sc, t, west, east, y, o, h, bad);
    if (more) {
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = hn[i];
      word = word_n;
    }
  }
}

// ---- shared-memory barriers and bulk copies (bounded waits) -----------------
__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// try_wait with a suspend-time hint: the thread sleeps in hardware until the
// phase completes or the hint (ns) elapses, instead of spinning
constexpr uint32_t kSuspendHintNs = 1000000;   // 1 ms per attempt

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

constexpr uint32_t kWaitLimit = 2000;   // attempts (x the 1 ms hint) before a wait gives up

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t k = 0; k < kWaitLimit; ++k)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// row index y wrapped into [0, ny) (y may lie any number of lattices away)
__device__ __forceinline__ int wrap_row(int y, int ny) {
  y %= ny;
  return y < 0 ? y + ny : y;
}

// ---- fused network blocks of the NN direct-reconstruction outflow -----------
// (Sec. 3.1, Eq. 15.)  Boundary blocks of the step launch rebuild the east
// fluid nodes of the members with a network outflow, concurrently with the
// stream-and-collide blocks: they read only the source buffer and write only
// the east column, which the other blocks leave to them.  With FP32 or FP16
// storage a block takes kNnTcNodes east nodes and runs the network on the
// tensor cores (nn_block_tc below).  With FP64 storage a block takes
// kNnNodes consecutive east nodes.  For each layer its warps split the
// inputs k: warp w sums its slice of k for every node and unit (lane j holds
// units j and j + 32; inputs are broadcast from shared memory; the transposed
// weights, row k = input k's weights to every unit, stream through L1 with
// coalesced loads), then the block adds the warps' partial sums in warp order.
constexpr int kNnNodes = 8;      // east nodes per network block
constexpr int kNnMaxW = 64;      // widest hidden layer

// shared memory of a network block: features, activations, per-warp partials
template <typename R>
constexpr size_t nn_smem_bytes(int warps) {
  return sizeof(R) * (size_t)kNnNodes * (81 + kNnMaxW + (size_t)warps * kNnMaxW);
}

template <typename S, typename R>
__device__ __forceinline__ R post_stream_h(const S* __restrict__ A, const Member& m, int x, int y,
                                           int i) {
  // post-stream, post-bounce-back h_i at node (x, y); y wraps
  y = y < 0 ? y + m.ny : (y >= m.ny ? y - m.ny : y);
  const bool solid = (__ldg(m.solid_bits + y * m.words_per_row + (x >> 5)) >> (x & 31)) & 1u;
  const int k = solid ? opp(i) : i;
  int sy = y - cy(k);
  sy = sy < 0 ? sy + m.ny : (sy >= m.ny ? sy - m.ny : sy);
  const int sx = x - cx(k);
  return to_r<R>(__ldcg(A + k * m.plane + sy * m.pitch + sx));
}

// ---- the network on the tensor cores (FP32 and FP16 storage) -----------------
// A block takes kNnTcNodes = 16 east nodes, the m-dimension of one mma tile.
// (1) One round of loads stages the window the block needs: the nine stored
// populations of columns L-4 .. L at rows y0-2 .. y0+17 (every pull of the
// 81 inputs of its nodes and of the nodes themselves) and the solid bits of
// those rows, while one thread copies the network blob (input constants and
// the weights, already split into TF32 high and low parts in fragment order:
// about 82 KB for 81-64-64-3) into shared memory with two cp.async.bulk
// copies (the constants first, the weights waited for only before layer 1).
// (2) The 81 inputs of every node are formed in shared memory (post-stream
// values: pulls, reversed at solid nodes; z-scored), zero-padded to K = 88 and
// stored as their TF32 high and low parts.  (3) Each layer is one GEMM
// [16 x K] x [K x N] with mma.sync m16n8k8 (3xTF32: hi*hi + hi*lo + lo*hi,
// FP32 accumulators initialised with the bias), which keeps the products to
// FP32 accuracy; the warps take the layer's 8-column n-tiles in turn, and a
// hidden layer's activations are stored split for the next.  (4) One thread
// per node applies Eq. 15 with the Zou & He fallback and collides.

// shared memory of a tensor-core network block: the network blob, then the
// window, solid bits, the high and low planes of the two activation tiles
// and the two copies' mbarriers
__host__ __device__ constexpr size_t nn_tc_fixed_bytes() {
  return (size_t)9 * kNnTcWin * 5 * 4 + 32 + 2 * (size_t)kNnTcNodes * kNnTcLdIn * 4 +
         2 * (size_t)kNnTcNodes * kNnTcLdAct * 4 + 2 * 8;
}
__host__ __device__ constexpr size_t nn_tc_smem_bytes(int blob_elems) {
  return (size_t)blob_elems * 4 + nn_tc_fixed_bytes();
}

// out[16][n_out] = act(in[16][n_in] W^T + b) for the block's 16 nodes.  in
// is given as its TF32 high and low planes (inH, inL; row stride ldi, zero
// past n_in up to a multiple of 8); wb is the layer's weights in fragment
// order (nn_tc_layer_floats), bias the padded bias.  A hidden layer writes
// its activations as high and low planes (outH, outL), the padded columns
// zero (zero weights and bias, act(0) = 0); the last layer writes plain
// values to outH.
__device__ inline void nn_layer_tc(const float* inH, const float* inL, int ldi, int n_in,
                                   float* outH, float* outL, int ldo, int n_out,
                                   const float* wb, const float* bias, bool hidden, int act) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
  const int g = lane >> 2, t4 = lane & 3;
  const int K8 = (n_in + 7) / 8, N8 = (n_out + 7) / 8;
  // this warp's n-tiles: warp and warp + nw (N8 <= 8 <= 2 nw: at most two)
  const int j0 = warp, j1 = warp + nw;
  const bool has0 = j0 < N8, has1 = j1 < N8;
  if (!has0) return;
  // per n-tile three accumulators: hi*hi (from the bias) and the two small
  // cross terms, so that each mma chain is one k-step long per k-step
  float c0[4], c1[4], p0[4] = {0.f, 0.f, 0.f, 0.f}, q0[4] = {0.f, 0.f, 0.f, 0.f};
  float p1[4] = {0.f, 0.f, 0.f, 0.f}, q1[4] = {0.f, 0.f, 0.f, 0.f};
  {
    const int nc0 = j0 * 8 + 2 * t4, nc1 = j1 * 8 + 2 * t4;
    c0[0] = c0[2] = bias[nc0];
    c0[1] = c0[3] = bias[nc0 + 1];
    c1[0] = c1[2] = has1 ? bias[nc1] : 0.f;
    c1[1] = c1[3] = has1 ? bias[nc1 + 1] : 0.f;
  }
  const float4* w0 = reinterpret_cast<const float4*>(wb) + (size_t)j0 * K8 * 32 + lane;
  const float4* w1 = reinterpret_cast<const float4*>(wb) + (size_t)j1 * K8 * 32 + lane;
#pragma unroll 2
  for (int kk = 0; kk < K8; ++kk) {
    const int k0 = kk * 8 + t4;
    uint32_t ah[4], al[4];
    ah[0] = __float_as_uint(inH[g * ldi + k0]);
    ah[1] = __float_as_uint(inH[(g + 8) * ldi + k0]);
    ah[2] = __float_as_uint(inH[g * ldi + k0 + 4]);
    ah[3] = __float_as_uint(inH[(g + 8) * ldi + k0 + 4]);
    al[0] = __float_as_uint(inL[g * ldi + k0]);
    al[1] = __float_as_uint(inL[(g + 8) * ldi + k0]);
    al[2] = __float_as_uint(inL[g * ldi + k0 + 4]);
    al[3] = __float_as_uint(inL[(g + 8) * ldi + k0 + 4]);
    {
      const float4 w = w0[kk * 32];
      mma_tf32_1688(p0, al, __float_as_uint(w.x), __float_as_uint(w.y));
      mma_tf32_1688(q0, ah, __float_as_uint(w.z), __float_as_uint(w.w));
      mma_tf32_1688(c0, ah, __float_as_uint(w.x), __float_as_uint(w.y));
    }
    if (has1) {
      const float4 w = w1[kk * 32];
      mma_tf32_1688(p1, al, __float_as_uint(w.x), __float_as_uint(w.y));
      mma_tf32_1688(q1, ah, __float_as_uint(w.z), __float_as_uint(w.w));
      mma_tf32_1688(c1, ah, __float_as_uint(w.x), __float_as_uint(w.y));
    }
  }
  // the small terms added first
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    c0[q] += p0[q] + q0[q];
    c1[q] += p1[q] + q1[q];
  }
  auto store = [&](const float c[4], int j) {
    const int nc = j * 8 + 2 * t4;
    const int idx[4] = {g * ldo + nc, g * ldo + nc + 1, (g + 8) * ldo + nc,
                        (g + 8) * ldo + nc + 1};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (hidden) {
        uint32_t hi, lo;
        tf32_split(act_hidden<float>(c[q], act), hi, lo);
        outH[idx[q]] = __uint_as_float(hi);
        outL[idx[q]] = __uint_as_float(lo);
      } else {
        outH[idx[q]] = c[q];
      }
    }
  };
  store(c0, j0);
  if (has1) store(c1, j1);
}

// The launch's dynamic shared memory seen from the boundary blocks: the same
// bytes as the kernels' own extern arrays, named here so that the compiler
// addresses them as shared memory (not through generic pointers).
extern __shared__ __align__(16) unsigned char ext_dyn_smem[];

template <typename S>
__device__ __noinline__ void nn_block_tc(const StepParams& p, const Member& m, int local_block,
                                         unsigned char*) {
  unsigned char* smem = ext_dyn_smem;
  constexpr int G = kNnTcNodes, WR = kNnTcWin;
  constexpr int NWIN = 9 * WR * 5;
  const int T = (int)blockDim.x;
  const int y0 = local_block * G;
  const int L = m.nx - 1;
  const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  float* net = reinterpret_cast<float*>(smem);                      // the network blob
  float* win = net + m.nn_blob_elems;                               // [9][WR][5]
  uint8_t* sol = reinterpret_cast<uint8_t*>(win + NWIN);            // [WR] solid bits of L-4 .. L
  float* buf0H = reinterpret_cast<float*>(sol + 32);                // [G][kNnTcLdIn], high
  float* buf0L = buf0H + G * kNnTcLdIn;                             // and low parts
  float* buf1H = buf0L + G * kNnTcLdIn;                             // [G][kNnTcLdAct]
  float* buf1L = buf1H + G * kNnTcLdAct;
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf1L + G * kNnTcLdAct);
  // (1) the network blob by two bulk copies overlapping the window loads:
  // the input constants (needed first, on bar[0]) and the weights (bar[1])
  constexpr uint32_t tab_bytes = 4u * kNnTcFeat * 4u;
  const uint32_t w_bytes = (uint32_t)m.nn_blob_elems * 4u - tab_bytes;
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_expect_tx(&bar[0], tab_bytes);
    bulk_copy_g2s(net, m.nn_net, tab_bytes, &bar[0]);
    mbar_expect_tx(&bar[1], w_bytes);
    bulk_copy_g2s(net + 4 * kNnTcFeat,
                  static_cast<const float*>(m.nn_net) + 4 * kNnTcFeat, w_bytes, &bar[1]);
  }
  // the window: A_i at rows y0-2+r, columns L-4+c; every load of a thread
  // issued before any is used
  {
    constexpr int Q = (NWIN + 127) / 128;
    float v[Q];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int e = (int)threadIdx.x + q * T;
      v[q] = 0.f;
      if (e < NWIN) {
        const int i = e / (WR * 5), r = (e / 5) % WR, c = e % 5;
        const int yy = wrap_row(y0 - 2 + r, m.ny);
        v[q] = to_r<float>(__ldcg(A + i * m.plane + yy * m.pitch + (L - 4 + c)));
      }
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int e = (int)threadIdx.x + q * T;
      if (e < NWIN) win[e] = v[q];
    }
  }
  if ((int)threadIdx.x < WR) {
    const int yy = wrap_row(y0 - 2 + (int)threadIdx.x, m.ny);
    const uint32_t* row = m.solid_bits + yy * m.words_per_row;
    const uint32_t lo = __ldg(row + ((L - 4) >> 5)), hi = __ldg(row + (L >> 5));
    uint32_t bits = 0;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int x = L - 4 + c;
      bits |= ((((x >> 5) == ((L - 4) >> 5) ? lo : hi) >> (x & 31)) & 1u) << c;
    }
    sol[threadIdx.x] = (uint8_t)bits;
  }
  // the constants must land before the inputs are formed: a bounded wait,
  // which on giving up latches DEV_TIMEOUT and waits once more so that no copy
  // is left in flight (the weights are waited for before the layers)
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar[0], 0)) {
    atomicOr(m.status, DEV_TIMEOUT);
    mbar_wait_bounded(&bar[0], 0);
  }
  __syncthreads();
  // post-stream h_i at window row r, column c (bounce-back at solid nodes)
  auto post = [&](int r, int c, int i) -> float {
    const bool solid = (sol[r] >> c) & 1u;
    const int k = solid ? opp(i) : i;
    return win[(k * WR + r - cy(k)) * 5 + c - cx(k)];
  };
  // (2) inputs, index k*27 + j*9 + i: column L-1-k, row y-1+j, population i;
  // a thread takes one input index for a quarter of the nodes, with its
  // z-score constants and window offsets read from the blob's table
  const float* tab = net;                       // [4][kNnTcFeat]
  constexpr int NQ = G / 4;
  for (int e = threadIdx.x; e < kNnTcFeat * 4; e += T) {
    const int kx = e % kNnTcFeat, n0 = (e / kNnTcFeat) * NQ;
    if (kx < 81) {
      const int j = (kx / 9) % 3, c = 3 - kx / 27;
      const float shift = tab[kx], inv = tab[kNnTcFeat + kx];
      const int off_f = (int)tab[2 * kNnTcFeat + kx];   // node fluid
      const int off_s = (int)tab[3 * kNnTcFeat + kx];   // node solid
#pragma unroll
      for (int n = n0; n < n0 + NQ; ++n) {
        const bool solid = (sol[n + j + 1] >> c) & 1u;
        uint32_t hi, lo;
        tf32_split((win[(solid ? off_s : off_f) + 5 * n] - shift) * inv, hi, lo);
        buf0H[n * kNnTcLdIn + kx] = __uint_as_float(hi);
        buf0L[n * kNnTcLdIn + kx] = __uint_as_float(lo);
      }
    } else {
#pragma unroll
      for (int n = n0; n < n0 + NQ; ++n) {
        buf0H[n * kNnTcLdIn + kx] = 0.f;
        buf0L[n * kNnTcLdIn + kx] = 0.f;
      }
    }
  }
  if (threadIdx.x == 0 && !mbar_wait_bounded(&bar[1], 0)) {
    atomicOr(m.status, DEV_TIMEOUT);
    mbar_wait_bounded(&bar[1], 0);
  }
  __syncthreads();
  // (3) the layers, alternating between the two tiles
  int off = 4 * kNnTcFeat;
  float *curH = buf0H, *curL = buf0L;
  int ld = kNnTcLdIn;
  for (int l = 0; l < m.nn_layers; ++l) {
    const int n_in = m.nn_sizes[l], n_out = m.nn_sizes[l + 1];
    const bool last = l == m.nn_layers - 1;
    float* nxtH = curH == buf0H ? buf1H : buf0H;
    float* nxtL = curH == buf0H ? buf1L : buf0L;
    const int wfl = nn_tc_layer_floats(n_in, n_out) - nn_tc_pad8(n_out);
    nn_layer_tc(curH, curL, ld, n_in, nxtH, nxtL, kNnTcLdAct, n_out, net + off, net + off + wfl,
                !last, m.nn_act);
    __syncthreads();
    off += nn_tc_layer_floats(n_in, n_out);
    curH = nxtH;
    curL = nxtL;
    ld = kNnTcLdAct;
  }
  const float* cur = curH;                      // the last layer's outputs (plain values)
  // (4) Eq. 15 with the Zou & He fallback, then collision; one thread per node
  const int n = threadIdx.x;
  const int y = y0 + n;
  if (n >= G || y >= m.ny) return;
  if ((sol[n + 2] >> 4) & 1u) return;   // a solid east node: the stream-and-collide blocks
  const Scalars<float> sc(m);
  // pulled populations of (L, y) from the window (those from x = L + 1 are rebuilt)
  float h[9];
  h[0] = win[(0 * WR + n + 2) * 5 + 4];
  h[1] = win[(1 * WR + n + 2) * 5 + 3];
  h[2] = win[(2 * WR + n + 1) * 5 + 4];
  h[4] = win[(4 * WR + n + 3) * 5 + 4];
  h[5] = win[(5 * WR + n + 1) * 5 + 3];
  h[8] = win[(8 * WR + n + 3) * 5 + 3];
  h[3] = h[6] = h[7] = 0.f;
  const float scale = (float)m.nn_out_scale;
  const float s3 = scale * cur[n * kNnTcLdAct + 0];
  const float s6 = scale * cur[n * kNnTcLdAct + 1];
  const float s7 = scale * cur[n * kNnTcLdAct + 2];
  float hn[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) hn[i] = h[i];
  // g_i(L) = f_i(L-1) + s_i, the bases taken post-stream at (L-1, y)
  hn[3] = post(n + 2, 3, 3) + s3;
  hn[6] = post(n + 2, 3, 6) + s6;
  hn[7] = post(n + 2, 3, 7) + s7;
  float drho_n, jx_n, jy_n;
  moments_shifted(hn, drho_n, jx_n, jy_n);
  bool ok = !nonfinite(s3) && !nonfinite(s6) && !nonfinite(s7);
  ok = ok && (hn[3] + wgt<float>(3) >= 0.f) && (hn[6] + wgt<float>(6) >= 0.f) &&
       (hn[7] + wgt<float>(7) >= 0.f);
  ok = ok && (fabsf((1.f + drho_n) - sc.rho_out) <= (float)m.nn_drho);
  if (ok) {
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = hn[i];
  } else {
    zouhe_east<float>(h, sc.rho_out);
    atomicAdd(m.nn_fallbacks, 1ull);
  }
  float drho, ux, uy;
  if (m.coll == LBM_BGK) collide_bgk<float>(h, sc.omega, drho, ux, uy);
  else collide_mrt<float>(h, mrt_of<float>(m), drho, ux, uy);
  if (nonfinite(drho)) atomicOr(m.status, DEV_NONFINITE);
  const int o = y * m.pitch + L;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[i]);
}

template <typename S>
__device__ __noinline__ void nn_block(const StepParams& p, const Member& m, int local_block,
                                      unsigned char* smem) {
  using R = typename Compute<S>::R;
  constexpr int G = kNnNodes;
  const int W = (int)(blockDim.x >> 5);
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int y0 = local_block * G;
  const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  const R* __restrict__ net = static_cast<const R*>(m.nn_net);
  const int L = m.nx - 1;
  R* feat = reinterpret_cast<R*>(smem);     // [G][81]
  R* act = feat + G * 81;                   // [G][kNnMaxW]
  R* red = act + G * kNnMaxW;               // [W][G][kNnMaxW]
  int n_params = 0;
  for (int l = 0; l < m.nn_layers; ++l)
    n_params += m.nn_sizes[l] * m.nn_sizes[l + 1] + m.nn_sizes[l + 1];
  const R* in_mean = net + n_params;
  const R* in_std = in_mean + 81;

  // the 81 z-scored inputs of each node (nodes past ny repeat the last row)
#pragma unroll 4
  for (int idx = threadIdx.x; idx < G * 81; idx += blockDim.x) {
    const int n = idx / 81, k = idx - n * 81;
    const int y = min(y0 + n, m.ny - 1);
    const int col = k / 27, j = (k / 9) % 3, i = k % 9;
    feat[idx] = (post_stream_h<S, R>(A, m, L - 1 - col, y + j - 1, i) + wgt<R>(i) -
                 ldg(in_mean + k)) / ldg(in_std + k);
  }
  __syncthreads();
  int off = 0;
  for (int l = 0; l < m.nn_layers; ++l) {
    const int n_in = m.nn_sizes[l], n_out = m.nn_sizes[l + 1];
    const R* __restrict__ Wt = net + off;
    const R* in = l == 0 ? feat : act;
    const int stride = l == 0 ? 81 : kNnMaxW;
    const int per = (n_in + W - 1) / W;
    const int k0 = wp * per, k1 = min(n_in, k0 + per);
    const int c0 = lane < n_out ? lane : 0;
    const int c1 = lane + 32 < n_out ? lane + 32 : 0;
    R acc[G][2];
#pragma unroll
    for (int n = 0; n < G; ++n) acc[n][0] = acc[n][1] = R(0);
#pragma unroll 8
    for (int k = k0; k < k1; ++k) {
      const R w0 = ldg(Wt + k * n_out + c0);
      const R w1 = ldg(Wt + k * n_out + c1);
#pragma unroll
      for (int n = 0; n < G; ++n) {
        const R xk = in[n * stride + k];
        acc[n][0] = fma(w0, xk, acc[n][0]);
        acc[n][1] = fma(w1, xk, acc[n][1]);
      }
    }
#pragma unroll
    for (int n = 0; n < G; ++n) {
      if (lane < n_out) red[(wp * G + n) * kNnMaxW + lane] = acc[n][0];
      if (lane + 32 < n_out) red[(wp * G + n) * kNnMaxW + lane + 32] = acc[n][1];
    }
    __syncthreads();
    const bool last = l == m.nn_layers - 1;
    const R* bias = Wt + n_in * n_out;
    for (int idx = threadIdx.x; idx < G * n_out; idx += blockDim.x) {
      const int n = idx / n_out, j = idx - n * n_out;
      R sum = ldg(bias + j);
      for (int w = 0; w < W; ++w) sum += red[(w * G + n) * kNnMaxW + j];
      act[n * kNnMaxW + j] = last ? sum : act_hidden<R>(sum, m.nn_act);
    }
    __syncthreads();
    off += n_in * n_out + n_out;
  }

  // Eq. 15 with the Zou & He fallback, then collision; one thread per node
  const int n = threadIdx.x;
  const int y = y0 + n;
  if (n >= G || y >= m.ny) return;
  if ((__ldg(m.solid_bits + y * m.words_per_row + (L >> 5)) >> (L & 31)) & 1u) return;
  const Scalars<R> sc(m);
  const int ym = y == 0 ? m.ny - 1 : y - 1;
  const int yp = y == m.ny - 1 ? 0 : y + 1;
  const int rc = y * m.pitch, rm = ym * m.pitch, rp = yp * m.pitch;
  const int xm = L - 1;
  // pulled populations (those from x = L + 1 are rebuilt below)
  R h[9];
  h[0] = to_r<R>(__ldcg(A + 0 * m.plane + rc + L));
  h[1] = to_r<R>(__ldcg(A + 1 * m.plane + rc + xm));
  h[2] = to_r<R>(__ldcg(A + 2 * m.plane + rm + L));
  h[3] = to_r<R>(__ldcg(A + 3 * m.plane + rc));
  h[4] = to_r<R>(__ldcg(A + 4 * m.plane + rp + L));
  h[5] = to_r<R>(__ldcg(A + 5 * m.plane + rm + xm));
  h[6] = to_r<R>(__ldcg(A + 6 * m.plane + rm));
  h[7] = to_r<R>(__ldcg(A + 7 * m.plane + rp));
  h[8] = to_r<R>(__ldcg(A + 8 * m.plane + rp + xm));
  const R scale = (R)m.nn_out_scale;
  const R s3 = scale * act[n * kNnMaxW + 0];
  const R s6 = scale * act[n * kNnMaxW + 1];
  const R s7 = scale * act[n * kNnMaxW + 2];
  R hn[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) hn[i] = h[i];
  // g_i(L) = f_i(L-1) + s_i, the bases taken post-stream at (L-1, y)
  hn[3] = post_stream_h<S, R>(A, m, L - 1, y, 3) + s3;
  hn[6] = post_stream_h<S, R>(A, m, L - 1, y, 6) + s6;
  hn[7] = post_stream_h<S, R>(A, m, L - 1, y, 7) + s7;
  R drho_n, jx_n, jy_n;
  moments_shifted(hn, drho_n, jx_n, jy_n);
  bool ok = !nonfinite(s3) && !nonfinite(s6) && !nonfinite(s7);
  ok = ok && (hn[3] + wgt<R>(3) >= R(0)) && (hn[6] + wgt<R>(6) >= R(0)) &&
       (hn[7] + wgt<R>(7) >= R(0));
  ok = ok && (fabs((R(1) + drho_n) - sc.rho_out) <= (R)m.nn_drho);
  if (ok) {
#pragma unroll
    for (int i = 0; i < 9; ++i) h[i] = hn[i];
  } else {
    zouhe_east<R>(h, sc.rho_out);
    atomicAdd(m.nn_fallbacks, 1ull);
  }
  R drho, ux, uy;
  if (m.coll == LBM_BGK) collide_bgk<R>(h, sc.omega, drho, ux, uy);
  else collide_mrt<R>(h, mrt_of<R>(m), drho, ux, uy);
  if (nonfinite(drho)) atomicOr(m.status, DEV_NONFINITE);
  const int o = rc + L;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[i]);
}

// ---- characteristic outflow blocks (Sec. 4, Eqs. 17-28) ----------------------
// One thread per east node (L, y), L = nx - 1; a block takes blockDim.x
// consecutive rows.  From the post-collision state at t (the source buffer):
// rho, u, v at (L, y), (L-1, y), (L-2, y), (L, y -+ 1); p = c_s^2 rho; d/dx
// second-order one-sided backward, d/dy central (periodic) or first-order
// towards the fluid next to a solid row.  The block first stages the moments of
// columns L-2 .. L for its rows and one row on each side in shared memory, each
// node computed once from loads of three adjacent columns (instead of every
// thread gathering 45 scattered populations).  Optional tuner: the six
// derivatives (p_x, u_x, v_x, p_y, u_y, v_y), z-scored, through a small MLP;
// sigma = sigma_max sigmoid(s_0), and with a second output kappa2 = kappa2_max
// sigmoid(s_1).  With FP32 or FP16 storage each warp evaluates the tuner for
// its 32 nodes on the tensor cores (BF16 operands, FP32 accumulation); with
// FP64 storage every thread evaluates it in FP64.  Wave amplitudes L5, L3
// (Eqs. 20-22), transverse terms T1, T3, T5 (Eqs. 23-25), incoming L1 of Eq. 26
// with kappa1 of Eq. 27, time derivatives (Eqs. 17-19) and one Euler step give
// the prescribed (rho, u, v) at t+1; the unknowns 3, 6, 7 of the post-stream
// node follow by Zou & He with that state and f_0 takes the correction of
// Eq. 28; then the node collides like any fluid node.
constexpr int kTunerMaxW = 32;    // widest hidden layer of the CBC tuner

template <typename R>
__device__ __forceinline__ R sigmoid_r(R s) { return R(1) / (R(1) + exp(-s)); }

// tuner outputs s[0..1] (s[1] = 0 with one output) for six inputs, one node
// per thread in the compute precision (the FP64 path)
template <typename R>
__device__ void tuner_eval(const Member& m, const R x_in[6], R s_out[2]) {
  const R* __restrict__ net = static_cast<const R*>(m.nn_net);
  int n_params = 0;
  for (int l = 0; l < m.nn_layers; ++l)
    n_params += m.nn_sizes[l] * m.nn_sizes[l + 1] + m.nn_sizes[l + 1];
  const R* in_mean = net + n_params;
  const R* in_std = in_mean + 6;
  R a[kTunerMaxW], b[kTunerMaxW];
  for (int k = 0; k < 6; ++k) a[k] = (x_in[k] - ldg(in_mean + k)) / ldg(in_std + k);
  int off = 0;
  for (int l = 0; l < m.nn_layers; ++l) {
    const int n_in = m.nn_sizes[l], n_out = m.nn_sizes[l + 1];
    const R* Wt = net + off;
    const bool last = l == m.nn_layers - 1;
    for (int j = 0; j < n_out; ++j) {
      R acc = ldg(Wt + n_in * n_out + j);
      for (int k = 0; k < n_in; ++k) acc = fma(ldg(Wt + k * n_out + j), a[k], acc);
      b[j] = last ? acc : act_hidden<R>(acc, m.nn_act);
    }
    for (int j = 0; j < n_out; ++j) a[j] = b[j];
    off += n_in * n_out + n_out;
  }
  s_out[0] = a[0];
  s_out[1] = m.nn_sizes[m.nn_layers] > 1 ? a[1] : R(0);
}

// ---- the tuner on the tensor cores (FP32 and FP16 storage) -------------------
// The 32 nodes of a warp form the rows of a [32 x K] activation tile; each
// layer is one warp-level GEMM with mma.sync m16n8k16 (BF16 operands, FP32
// accumulators initialised with the bias), two m-tiles of 16 nodes.  Layer
// widths are padded: the six inputs to K = 16, hidden widths to 16 or 32 (at
// most 32, so at most 4 n-tiles and 2 k-steps), the last layer to N = 8.  The
// accumulator fragment of two neighbouring n-tiles is exactly the A fragment of
// the next layer's k-step, so activations stay in registers between layers
// (padded columns hold 0: zero weights and bias, and act(0) = 0).  The weights
// come from the library's padded BF16 copy ([N_pad][K_pad] per layer, K
// fastest), biases from the FP32 copy.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);   // lo in the low half
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__host__ __device__ constexpr int tuner_pad16(int n) { return (n + 15) / 16 * 16; }

// per-warp shared scratch of the tensor-core tuner: [32][8] BF16 inputs, [32][2] outputs
constexpr int kTunerWarpBytes = 32 * 8 * 2 + 32 * 2 * 4;

// z: this thread's six z-scored inputs; every lane of the warp must call it.
__device__ inline void tuner_mma_warp(const Member& m, const float z[6], float s_out[2],
                               unsigned char* wscratch) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  uint32_t* feat = reinterpret_cast<uint32_t*>(wscratch);          // [32][4] bf16 pairs
  float* outs = reinterpret_cast<float*>(wscratch + 32 * 8 * 2);   // [32][2]
  feat[lane * 4 + 0] = pack_bf16x2(z[0], z[1]);
  feat[lane * 4 + 1] = pack_bf16x2(z[2], z[3]);
  feat[lane * 4 + 2] = pack_bf16x2(z[4], z[5]);
  feat[lane * 4 + 3] = 0u;
  __syncwarp();
  const uint16_t* __restrict__ W = static_cast<const uint16_t*>(m.nn_bf16);
  const float* __restrict__ net = static_cast<const float*>(m.nn_net);
  const int L = m.nn_layers;
#pragma unroll 1
  for (int mt = 0; mt < 2; ++mt) {
    const int ra = mt * 16 + g, rb = ra + 8;
    uint32_t a[2][4];
    a[0][0] = feat[ra * 4 + t4];
    a[0][1] = feat[rb * 4 + t4];
    a[0][2] = a[0][3] = 0u;
    a[1][0] = a[1][1] = a[1][2] = a[1][3] = 0u;
    int ksteps = 1, woff = 0, foff = 0;
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      const int n_in = m.nn_sizes[l], n_out = m.nn_sizes[l + 1];
      const bool last = l == L - 1;
      const int Kp = l == 0 ? 16 : tuner_pad16(n_in);
      const int Np = last ? 8 : tuner_pad16(n_out);
      const int nt = Np / 8;
      const float* bias = net + foff + n_in * n_out;
      float c[4][4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        c[j][0] = c[j][1] = c[j][2] = c[j][3] = 0.f;
        if (j < nt) {
          const int n0 = j * 8 + 2 * t4;
          const float b0 = n0 < n_out ? __ldg(bias + n0) : 0.f;
          const float b1 = n0 + 1 < n_out ? __ldg(bias + n0 + 1) : 0.f;
          c[j][0] = b0;
          c[j][1] = b1;
          c[j][2] = b0;
          c[j][3] = b1;
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            if (kk < ksteps) {
              const uint16_t* wr = W + woff + (j * 8 + g) * Kp + kk * 16 + 2 * t4;
              const uint32_t b0r = __ldg(reinterpret_cast<const unsigned int*>(wr));
              const uint32_t b1r = __ldg(reinterpret_cast<const unsigned int*>(wr + 8));
              mma_bf16_16816(c[j], a[kk], b0r, b1r);
            }
          }
        }
      }
      if (!last) {
        ksteps = Np / 16;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          if (kk < ksteps) {
            const int j0 = 2 * kk, j1 = 2 * kk + 1;
            a[kk][0] = pack_bf16x2(act_hidden<float>(c[j0][0], m.nn_act),
                                   act_hidden<float>(c[j0][1], m.nn_act));
            a[kk][1] = pack_bf16x2(act_hidden<float>(c[j0][2], m.nn_act),
                                   act_hidden<float>(c[j0][3], m.nn_act));
            a[kk][2] = pack_bf16x2(act_hidden<float>(c[j1][0], m.nn_act),
                                   act_hidden<float>(c[j1][1], m.nn_act));
            a[kk][3] = pack_bf16x2(act_hidden<float>(c[j1][2], m.nn_act),
                                   act_hidden<float>(c[j1][3], m.nn_act));
          }
        }
      } else if (t4 == 0) {
        // columns 0 and 1 of n-tile 0: s_0, s_1 of rows ra and rb
        outs[ra * 2] = c[0][0];
        outs[ra * 2 + 1] = c[0][1];
        outs[rb * 2] = c[0][2];
        outs[rb * 2 + 1] = c[0][3];
      }
      woff += Np * Kp;
      foff += n_in * n_out + n_out;
    }
  }
  __syncwarp();
  s_out[0] = outs[lane * 2];
  s_out[1] = m.nn_sizes[L] > 1 ? outs[lane * 2 + 1] : 0.f;
}

// Rows (east nodes) of one CBC block of `threads` threads: every thread
// stages one row of the window, which reaches one row beyond the block's
// nodes on each side.
__host__ __device__ constexpr int cbc_block_rows(int threads) { return threads - 2; }

// shared memory of a CBC block of `threads` threads: per window row the
// moments of columns L-2, L-1, L ([3][rho - 1, u, v]) and six stored
// populations (A_0, A_2, A_4 at L; A_1, A_5, A_8 at L-1: the known pulls of the
// east node), then (FP32 compute) the per-warp scratch of the tensor-core tuner
template <typename R>
__host__ __device__ constexpr size_t cbc_win_bytes(int threads) {
  return ((size_t)threads * 15 * sizeof(R) + 15) / 16 * 16;
}
template <typename R>
__host__ __device__ constexpr size_t cbc_smem_bytes(int threads) {
  return cbc_win_bytes<R>(threads) + (sizeof(R) == 4 ? (size_t)(threads / 32) * kTunerWarpBytes : 0);
}

template <typename S>
__device__ __noinline__ void cbc_block(const StepParams& p, const Member& m, int local_block,
                                       unsigned char*) {
  using R = typename Compute<S>::R;
  unsigned char* smem = ext_dyn_smem;
  const int T = (int)blockDim.x;
  const int E = cbc_block_rows(T);
  const int t = (int)threadIdx.x;
  const int y0 = local_block * E;   // nodes y0 .. y0 + E - 1 on threads 1 .. E
  const int L = m.nx - 1;
  auto solid = [&](int x, int yy) -> bool {
    return (__ldg(m.solid_bits + yy * m.words_per_row + (x >> 5)) >> (x & 31)) & 1u;
  };
  const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  R* mac = reinterpret_cast<R*>(smem);   // [T][3 columns][rho - 1, u, v]
  R* raw = mac + 9 * T;                  // [T][A_0, A_2, A_4 at L; A_1, A_5, A_8 at L-1]
  {
    // window row t is lattice row y0 - 1 + t (wrapped): its 27 stored
    // populations of columns L-2 .. L, all loads issued before any is used
    const S* src = A + wrap_row(y0 - 1 + t, m.ny) * m.pitch + (L - 2);
    R v[9][3];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[i][c] = to_r<R>(__ldcg(src + i * m.plane + c));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const R h[9] = {v[0][c], v[1][c], v[2][c], v[3][c], v[4][c],
                      v[5][c], v[6][c], v[7][c], v[8][c]};
      R d, jx, jy;
      moments_shifted(h, d, jx, jy);
      const R rho = R(1) + d;
      mac[9 * t + 3 * c] = d;
      mac[9 * t + 3 * c + 1] = jx / rho;
      mac[9 * t + 3 * c + 2] = jy / rho;
    }
    raw[6 * t] = v[0][2];
    raw[6 * t + 1] = v[2][2];
    raw[6 * t + 2] = v[4][2];
    raw[6 * t + 3] = v[1][1];
    raw[6 * t + 4] = v[5][1];
    raw[6 * t + 5] = v[8][1];
  }
  __syncthreads();
  // threads 0 and T-1 (halo rows) and nodes past the last row compute on a
  // neighbouring row and write nothing: every lane of a warp takes part in the
  // tensor-core tuner
  const int tc = t < 1 ? 1 : (t > E ? E : t);   // window row of the node this thread evaluates
  const int y = y0 + tc - 1;
  const int yy = y < m.ny ? y : m.ny - 1;
  const bool active = t == tc && y < m.ny && !solid(L, yy);
  const int ym = yy == 0 ? m.ny - 1 : yy - 1;
  const int yp = yy == m.ny - 1 ? 0 : yy + 1;
  const R* w0 = mac + 9 * tc;
  const bool s_dn = solid(L, ym), s_up = solid(L, yp);
  const R cs2 = R(1) / R(3);
  const R cs = sqrt(cs2);
  // the stencil's values and derivatives from the staged window (row y - 1 at
  // w0 - 9, row y + 1 at w0 + 9); r* hold rho - 1 and p - 1/3 = c_s^2 (rho - 1).
  // Evaluated before the tuner for its features and again after it, so the
  // tuner's fragments do not compete with them for registers.
  struct Stencil { R r0, u0, v0, px, ux, vx, py, uy, vy; };
  auto stencil = [&]() {
    Stencil st;
    const R* wm = w0 - 9;
    const R* wp = w0 + 9;
    st.r0 = w0[6];
    st.u0 = w0[7];
    st.v0 = w0[8];
    st.px = cs2 * (R(0.5) * (R(3) * st.r0 - R(4) * w0[3] + w0[0]));
    st.ux = R(0.5) * (R(3) * st.u0 - R(4) * w0[4] + w0[1]);
    st.vx = R(0.5) * (R(3) * st.v0 - R(4) * w0[5] + w0[2]);
    auto ddy = [&](R qm, R q0, R qp) -> R {
      if (!s_up && !s_dn) return R(0.5) * (qp - qm);
      if (!s_up) return qp - q0;
      if (!s_dn) return q0 - qm;
      return R(0);
    };
    st.py = cs2 * ddy(wm[6], st.r0, wp[6]);
    st.uy = ddy(wm[7], st.u0, wp[7]);
    st.vy = ddy(wm[8], st.v0, wp[8]);
    return st;
  };
  R sigma = (R)m.cbc_sigma, kappa2 = (R)m.cbc_kappa2;
  if (m.nn_layers > 0) {   // block-uniform
    R s[2];
    {
      const Stencil f = stencil();
      const R feats[6] = {f.px, f.ux, f.vx, f.py, f.uy, f.vy};
      if constexpr (sizeof(R) == 4) {
        const float* net = static_cast<const float*>(m.nn_net);
        int n_params = 0;
        for (int l = 0; l < m.nn_layers; ++l)
          n_params += m.nn_sizes[l] * m.nn_sizes[l + 1] + m.nn_sizes[l + 1];
        float z[6];
#pragma unroll
        for (int k = 0; k < 6; ++k)
          z[k] = (feats[k] - __ldg(net + n_params + k)) / __ldg(net + n_params + 6 + k);
        tuner_mma_warp(m, z, s, smem + cbc_win_bytes<R>(T) + (t >> 5) * kTunerWarpBytes);
      } else {
        tuner_eval<R>(m, feats, s);
      }
    }
    sigma = sigma * sigmoid_r(s[0]);
    if (m.nn_sizes[m.nn_layers] > 1) kappa2 = kappa2 * sigmoid_r(s[1]);
  }
  if (!active) return;   // the stream-and-collide blocks handle solid nodes
  const Stencil st = stencil();
  const R r0 = st.r0, u0 = st.u0, v0 = st.v0, px = st.px, ux = st.ux, vx = st.vx;
  const R py = st.py, vy = st.vy;
  // Eqs. 20-27 and the Euler step of Eqs. 17-19
  const R rho = R(1) + r0;
  const R pL = cs2 * rho;
  const R L5 = (u0 + cs) * (px + rho * cs * ux);
  const R L3 = u0 * vx;
  const R T1 = -(v0 * py + pL * vy - rho * cs * v0 * vy);
  const R T3 = -(v0 * vy + py / rho);
  const R T5 = -(v0 * py + pL * vy + rho * cs * v0 * vy);
  const R kappa1 = sigma * (R)m.cbc_kfac;
  const R L1 = kappa1 * (cs2 * (r0 - (R)(m.rho_out - 1.0))) - kappa2 * T1 + T1;
  const R dr = r0 + (-(L5 + L1) / (R(2) * cs2) + (T5 + T1) / (R(2) * cs2));   // rho - 1 at t+1
  const R un = u0 + (-(L5 - L1) / (R(2) * rho * cs) + (T5 - T1) / (R(2) * rho * cs));
  const R vn = v0 + (-L3 + T3);
  // post-stream node: the known pulls from the window (those from x = L + 1
  // are rebuilt below)
  R h[9];
  h[0] = raw[6 * tc];
  h[2] = raw[6 * (tc - 1) + 1];
  h[4] = raw[6 * (tc + 1) + 2];
  h[1] = raw[6 * tc + 3];
  h[5] = raw[6 * (tc - 1) + 4];
  h[8] = raw[6 * (tc + 1) + 5];
  // Zou & He with the prescribed state, then Eq. 28 on f_0
  const R sknown = (h[0] + h[2] + h[4]) + R(2) * (h[1] + h[5] + h[8]);   // rho0 + 2 rho+ - 1
  R heq[9];
  heq_sym(dr, un, vn, heq);
  const R half_t = R(0.5) * ((h[4] - heq[4]) - (h[2] - heq[2]));
  h[3] = heq[3] + (h[1] - heq[1]);
  h[6] = heq[6] + (h[8] - heq[8]) + half_t;
  h[7] = heq[7] + (h[5] - heq[5]) - half_t;
  const R excess = dr + un + dr * un - sknown;          // rho (1 + u) - (rho0 + 2 rho+)
  h[0] += m.cbc_exact ? excess : excess / (R(1) + un);
  const Scalars<R> sc(m);
  R drho, uxo, uyo;
  if (m.coll == LBM_BGK) collide_bgk<R>(h, sc.omega, drho, uxo, uyo);
  else collide_mrt<R>(h, mrt_of<R>(m), drho, uxo, uyo);
  if (nonfinite(drho)) atomicOr(m.status, DEV_NONFINITE);
  const int o = y * m.pitch + L;
#pragma unroll
  for (int i = 0; i < 9; ++i) B[i * m.plane + o] = from_r<S>(h[i]);
}

// the network block of the storage precision: tensor cores for FP32 / FP16,
// FP64 on the FP64 pipe
template <typename S>
__device__ __forceinline__ void nn_dispatch(const StepParams& p, const Member& m, int blk,
                                            unsigned char* smem) {
  if constexpr (sizeof(typename Compute<S>::R) == 4) nn_block_tc<S>(p, m, blk, smem);
  else nn_block<S>(p, m, blk, smem);
}

template <typename S>
__device__ __forceinline__ void ext_dispatch(const StepParams& p, int blk, unsigned char* smem) {
  if (p.n_members == 1) {
    if (p.m0.ext_kind == 1) nn_dispatch<S>(p, p.m0, blk, smem);
    else cbc_block<S>(p, p.m0, blk, smem);
    return;
  }
  // the block's member record staged in shared memory once (coalesced), so
  // the boundary code reads its fields without global round trips
  __shared__ __align__(16) Member s_ext;
  constexpr int kWords = (int)(sizeof(Member) / sizeof(uint64_t));
  if (threadIdx.x < 32) {
    const uint64_t* src = reinterpret_cast<const uint64_t*>(p.members + p.nn_block_member[blk]);
    uint64_t* dst = reinterpret_cast<uint64_t*>(&s_ext);
    for (int w = threadIdx.x; w < kWords; w += 32) dst[w] = src[w];
  }
  __syncthreads();
  const int local = blk - s_ext.nn_first;
  if (s_ext.ext_kind == 1) nn_dispatch<S>(p, s_ext, local, smem);
  else cbc_block<S>(p, s_ext, local, smem);
}

// Block roles of a step launch: first one force-reduction block per member
// (they sum the previous step's partials and finish within microseconds),
// then the stream-and-collide and boundary blocks in the order of the launch
// table p.launch_order (entry v >= 0: stream-and-collide block v; v < 0:
// boundary block -v - 1), or, without boundary blocks, the stream-and-collide
// blocks in order.  The host places each boundary block next to the strips of
// its lattice's east tile that cover its rows, so the two read (and write)
// the same sectors of the east columns while they are in L2, instead of each
// fetching them from DRAM; when the whole grid is resident at once (or on the
// resident-sized grids, whose blocks live for the whole step) the boundary
// blocks come first, where their longer dependent chains start at once.
enum : int { ROLE_REDUCE = 0, ROLE_BOUNDARY = 1, ROLE_BULK = 2 };
struct BlockRole {
  int kind, idx;
};
__device__ __forceinline__ BlockRole block_role(const StepParams& p) {
  const int g = (int)blockIdx.x;
  if (g < p.n_members) return {ROLE_REDUCE, g};
  const int r = g - p.n_members;
  if (!p.launch_order) return {ROLE_BULK, r};
  const int v = __ldg(p.launch_order + r);
  return v >= 0 ? BlockRole{ROLE_BULK, v} : BlockRole{ROLE_BOUNDARY, -v - 1};
}

template <typename S, int COLL, int MINB, bool EXT>
__global__ void __launch_bounds__(128, MINB) step_kernel(const StepParams p) {
  using R = typename Compute<S>::R;
  extern __shared__ __align__(16) unsigned char nn_smem[];   // boundary blocks only
  pdl_launch_dependents();
  pdl_wait();
  const BlockRole role = block_role(p);
  if (EXT && role.kind == ROLE_BOUNDARY) {
    ext_dispatch<S>(p, role.idx, nn_smem);
    return;
  }
  const int64_t t = step_index(p);
  if (role.kind == ROLE_REDUCE) {
    if (p.reduce_prev && t >= 1) reduce_force(p, role.idx, t - 1);
    return;
  }
  const int b = role.idx;   // stream-and-collide block
  const int nblocks = (int)gridDim.x - p.nn_blocks - p.n_members;
  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;
  if (p.n_members == 1) {
    // the member lives in the parameter bank: no registers held for its fields
    const Scalars<R> sc(p.m0);
    const int strips = p.m0.strip_count;
    const int stride = p.persistent ? nblocks : strips;
    for (int s = b; s < strips; s += stride)
      reg_strip<S, COLL>(p, p.m0, sc, t, s, fx, fy, touched, bad);
    write_partial(p, t, b, fx, fy, touched, bad, p.m0.status);
  } else {
    const int sg = p.strip_order ? p.strip_order[b] : b;   // strips holding solids first
    const Member& m = p.members[p.strip_member[sg]];
    const Scalars<R> sc(m);
    reg_strip<S, COLL>(p, m, sc, t, sg - m.strip_first, fx, fy, touched, bad);
    write_partial(p, t, p.strip_force ? p.strip_force[sg] : sg, fx, fy, touched, bad, m.status);
  }
}

// ---- bulk-copy staged kernel -------------------------------------------------
// One block = one strip.  Thread 0 stages, for each output row, the nine
// source row segments (rows y - c_iy, columns shifted by -c_ix) plus the row's
// solid-mask words into a ring of NS shared-memory slots with cp.async.bulk
// copies that complete on one mbarrier per slot; all threads collide from
// shared memory and store coalesced rows.  Each staged segment starts A
// elements (16 bytes) before the tile, so every copy is 16-byte aligned and
// the x shifts become fixed offsets.  Waits are bounded: a wait that gives up
// latches DEV_TIMEOUT and the block drains its copies before it exits.

size_t step_bulk_smem(int prec, int stages);   // dynamic shared memory of the staged kernel

template <typename S>
struct BulkLayout {
  static constexpr int A = 16 / (int)sizeof(S);      // 16 bytes in elements
  static constexpr int SEG = 128 + A;                // staged elements per source row
  static constexpr int SEG_BYTES = SEG * (int)sizeof(S);
  static constexpr int STAGE_BYTES = 9 * SEG_BYTES + 16;   // + 4 solid-mask words
  static constexpr uint32_t TX_BYTES = (uint32_t)STAGE_BYTES;
};


constexpr int kConsumerWarps = 4;
constexpr int kBulkThreads = 32 * (kConsumerWarps + 1);

// ---- dataflow around the east boundary blocks --------------------------------
// With the NN or characteristic outflow a launch also holds boundary blocks:
// block j of a member rebuilds the east fluid nodes of rows [j e, (j+1) e),
// e = kNnNodes (NN) or the block size (CBC), reading the source columns
// L-4 .. L of rows y0-2 .. y1+2 (NN features are pulled populations of three
// columns and rows; the CBC stencil is narrower) and writing column L.  Their
// flags follow the strips' (p.ext_flags + the block's index in the launch).
// A boundary block of step t waits for the strips of the east tiles and the
// boundary blocks of step t-1 that meet its rows +- 2; a strip of an east
// tile (one that holds a column in L-4 .. L) also waits for the boundary
// blocks of step t-1 that meet its rows +- 2 (they wrote its column L, and read
// what it overwrites).

// Calls fn(s, e) for the wrapped row segments [s, e] covering rows a..b.
template <typename F>
__device__ __forceinline__ void row_segments(int a, int b, int ny, F fn) {
  if (b - a + 1 >= ny) {
    fn(0, ny - 1);
    return;
  }
  const int s = wrap_row(a, ny), e = wrap_row(b, ny);
  if (s <= e) {
    fn(s, e);
  } else {
    fn(s, ny - 1);
    fn(0, e);
  }
}

// rows of one boundary block of member m
__device__ __forceinline__ int ext_rows(const Member& m) { return m.ext_rows; }

// One poll: have the east-tile strips (if `strips`) and the boundary blocks (if
// `exts`) of member m whose rows meet a..b completed t steps?
__device__ inline bool east_ready(const StepParams& p, const Member& m, int a, int b, int64_t t,
                                 bool strips, bool exts) {
  bool ok = true;
  const int L = m.nx - 1;
  const int c0 = (L >= 4 ? L - 4 : 0) >> 7, c1 = L >> 7;
  const int per = ext_rows(m);
  row_segments(a, b, m.ny, [&](int s, int e) {
    if (exts) {
      const int64_t* f = p.strip_done + p.ext_flags + m.nn_first;
#pragma unroll 4
      for (int j = s / per; j <= e / per; ++j) ok &= ld_relaxed(f + j) >= t;
    }
    if (strips) {
      for (int r = s / p.rows; r <= e / p.rows; ++r)
        for (int c = c0; c <= c1; ++c)
          ok &= ld_relaxed(p.strip_done + m.strip_first + r * m.tiles_x + c) >= t;
    }
  });
  return ok;
}

// Bounded wait for east_ready; the fence after the last poll makes it an acquire.
__device__ inline bool wait_east(const StepParams& p, const Member& m, int a, int b, int64_t t,
                                 bool strips, bool exts) {
  uint64_t t0 = 0;
  for (uint32_t k = 0; k < (1u << 24); ++k) {
    if (east_ready(p, m, a, b, t, strips, exts)) {
      __threadfence();
      return true;
    }
    if (k == 0) t0 = global_ns();
    else if (global_ns() - t0 > kFlagWaitNs || timed_out_already(m.status)) break;
    __nanosleep(200);
  }
  __threadfence();
  return false;
}

// ---- row-window staging (variants 3, 4, 6) -----------------------------------
// A slot of the ring holds one input row of all nine populations: columns
// x0 - A .. x0 + 127 + A of the strip's tile (A = 16 bytes in elements, so the
// copy starts on a 16-byte boundary; columns outside the lattice read zeros
// and are never used), fetched by one 3-D tensor copy (x, y, population) of a
// W x 1 x 9 box, plus the row's 16 bytes of solid-mask words.  Output row y
// pulls population i from input row y - c_iy at column x - c_ix, so it reads
// three consecutive slots; each input row is copied once per strip.
template <typename S>
struct WinLayout {
  static constexpr int A = 16 / (int)sizeof(S);
  static constexpr int W = 128 + 2 * A;                    // staged columns
  static constexpr int ROW_BYTES = 9 * W * (int)sizeof(S);
  static constexpr int SLOT_BYTES = (ROW_BYTES + 16 + 127) / 128 * 128;
  static constexpr uint32_t TX_BYTES = (uint32_t)ROW_BYTES + 16u;
};

// One W x 1 x 9 box of a population buffer (its tensor map: x, y,
// population) into shared memory, completing on bar.  x * sizeof(S) must be a
// multiple of 16 (x may be negative: those columns read zeros).
__device__ __forceinline__ void tma_row_g2s(void* dst, const void* tmap, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(0), "r"(smem_u32(bar))
      : "memory");
}

// One node after its nine pulled values are loaded: the periodic wrap of the
// x +- 1 neighbours at the lattice edges, then bounce-back with momentum
// exchange, or the boundary condition and the collision.
template <typename S, int COLL>
__device__ __forceinline__ void finish_node(const Member& m, const Scalars<typename Compute<S>::R>& sc,
                                            const S* A, S* B, int x, int y, bool solid,
                                            int64_t t, typename Compute<S>::R h[9], double& fx,
                                            double& fy, bool& touched, bool& bad) {
  using R = typename Compute<S>::R;
  const int nx = m.nx, ny = m.ny, plane = m.plane, pitch = m.pitch;
  if (x == 0 || x == nx - 1) {
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    // (A is not __restrict__: these plain loads must not take the
    // non-coherent path, the previous launch may still be writing A)
    if (x == 0) {
      h[1] = to_r<R>(A[1 * plane + y * pitch + nx - 1]);
      h[5] = to_r<R>(A[5 * plane + ym * pitch + nx - 1]);
      h[8] = to_r<R>(A[8 * plane + yp * pitch + nx - 1]);
    }
    if (x == nx - 1) {
      h[3] = to_r<R>(A[3 * plane + y * pitch]);
      h[6] = to_r<R>(A[6 * plane + ym * pitch]);
      h[7] = to_r<R>(A[7 * plane + yp * pitch]);
    }
  }
  const bool west = !m.x_periodic && x == 0;
  const bool east = !m.x_periodic && x == nx - 1;
  const int o = y * pitch + x;
  // the network blocks rebuild external east fluid nodes; solid ones stay here
  if (solid)
    solid_node<S, R>(A, B, m, x, y, o, h, fx, fy, touched);
  else if (!(east && m.east_mode == EAST_EXTERNAL))
    fluid_node<S, R, COLL>(B, m, sc, t, west, east, y, o, h, bad);
}

// One block streams the rows of its strips (local strips lb, lb + gk, ... of
// member m) through an NS-slot ring of input rows with warp specialisation:
// warp 4 is the producer -- its lane 0 waits until a slot is released
// ("empty" barrier, one arrival per consumer warp), then fetches the next
// input row (rows y0 - 1 .. y0 + nrows of each strip, wrapped) with one tensor
// copy and one bulk copy completing on the slot's "full" barrier -- and warps
// 0-3 are consumers: for output row y each waits for input row y + 1, collides
// its 32 columns from input rows y - 1, y, y + 1 and releases row y - 1.  No
// block-wide barrier per row: warps run ahead independently.
template <typename S, int COLL, int NS>
__device__ __forceinline__ void bulk_run_window(const StepParams& p, const Member& m, int lb,
                                                int gk, unsigned char* smem_base) {
  static_assert(NS >= 3, "an output row needs three input rows in the ring");
  using R = typename Compute<S>::R;
  using Lay = WinLayout<S>;
  // the ring is 128-byte aligned (tensor copies); barriers after the slots
  unsigned char* smem = smem_base + ((128u - (smem_u32(smem_base) & 127u)) & 127u);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * Lay::SLOT_BYTES);
  uint64_t* empty = full + NS;
  __shared__ int s_abort;
  const S* A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  const void* tmap = m.tmap[p.q];
  const int nx = m.nx, ny = m.ny, tiles_x = m.tiles_x, rows = p.rows;
  const int strips = m.strip_count;
  const int warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int64_t t = step_index(p);
  const bool flow = p.strip_done != nullptr;   // one strip per block (variant 6)
  if (p.strip_done && threadIdx.x == kConsumerWarps * 32) {
    // the producer lane: wait for the strips around this one (and, in an east
    // tile, the boundary blocks next to it) to complete step t-1; the fence
    // orders those acquires before its copies (async proxy)
    bool ok = wait_strip_neighbours(p, m, lb, t);
    const int c = lb % m.tiles_x, L = m.nx - 1;
    if (ok && m.ext_kind != 0 && (c << 7) + 127 >= L - 4) {
      const int y0 = (lb / m.tiles_x) * p.rows;
      ok = wait_east(p, m, y0 - 2, min(y0 + p.rows, m.ny) + 1, t, false, true);
    }
    if (!ok) atomicOr(m.status, DEV_TIMEOUT);
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();
  // set-up done: wait for the previous step to complete before touching the
  // populations (it may still be reading the buffer this step writes)
  if (!flow) pdl_wait();

  // strip geometry
  struct Strip {
    int y0, x0, nrows;
  };
  auto strip_at = [&](int ls) {
    Strip st;
    st.y0 = (ls / tiles_x) * rows;
    st.x0 = (ls % tiles_x) << 7;
    st.nrows = min(rows, ny - st.y0);
    return st;
  };

  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if ((threadIdx.x & 31) == 0) {
      // input row k goes to slot k mod NS; its "empty" wait is for the
      // slot's previous use (phase of round k / NS - 1)
      int ps = lb, pr = -1, k = 0, slot = 0;
      uint32_t round = 0;
      Strip pst = strip_at(lb);
      while (ps < strips) {
        if (k >= NS && !mbar_wait_bounded(&empty[slot], (round - 1) & 1u)) {
          atomicOr(m.status, DEV_TIMEOUT);
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        int y = pst.y0 + pr;                    // input rows y0 - 1 .. y0 + nrows, wrapped
        y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
        unsigned char* st = smem + slot * Lay::SLOT_BYTES;
        if (pr >= 0 && pr < pst.nrows) {
          // a row of the strip: all nine populations and its solid-mask words
          mbar_expect_tx(&full[slot], Lay::TX_BYTES);
          tma_row_g2s(st, tmap, pst.x0 - Lay::A, y, &full[slot]);
          bulk_copy_g2s(st + Lay::ROW_BYTES,
                        m.solid_bits + y * m.words_per_row + (pst.x0 >> 5), 16u, &full[slot]);
        } else {
          // a halo row: only the three populations pulled across the strip's
          // edge (c_iy = 1 from the row above it, c_iy = -1 from the row
          // below); at x0 = 0 the copy starts at the lattice's first column
          const int lead = pst.x0 == 0 ? 0 : Lay::A;
          const uint32_t bytes = (uint32_t)((Lay::W - Lay::A + lead) * (int)sizeof(S));
          mbar_expect_tx(&full[slot], 3u * bytes);
          const int i0 = pr < 0 ? 2 : 4;       // 2, 5, 6 or 4, 7, 8
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            const int i = j == 0 ? i0 : i0 + 3 + (j - 1);
            bulk_copy_g2s(st + (i * Lay::W + Lay::A - lead) * (int)sizeof(S),
                          A + i * m.plane + y * m.pitch + pst.x0 - lead, bytes, &full[slot]);
          }
        }
        ++k;
        if (++slot == NS) {
          slot = 0;
          ++round;
        }
        if (++pr == pst.nrows + 1) {
          pr = -1;
          ps += gk;
          if (ps < strips) pst = strip_at(ps);
        }
      }
      // no copy may land after the block exits: wait (bounded) for the last
      // item staged into each slot
      for (int kk = k > NS ? k - NS : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NS], (uint32_t)((kk / NS) & 1));
    }
  } else {
    // ---------------- consumers ----------------
    const Scalars<R> sc(m);
    const int lx = threadIdx.x;     // column within the 128-wide tile
    const int lane = threadIdx.x & 31;
    // ring position of input row k as (slot, phase), advanced one row at a time
    struct Pos {
      int slot;
      uint32_t phase;
    };
    auto next = [](Pos q) {
      return ++q.slot == NS ? Pos{0, q.phase ^ 1u} : q;
    };
    auto wait_full = [&](Pos q) {
      // warp-uniform outcome, so the warp never diverges around __syncwarp
      return __all_sync(0xffffffffu, !s_abort && mbar_wait_bounded(&full[q.slot], q.phase));
    };
    auto release = [&](Pos q) {
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[q.slot]))
                     : "memory");
    };
    auto row_at = [&](Pos q) {
      return reinterpret_cast<const S*>(smem + q.slot * Lay::SLOT_BYTES);
    };
    bool ok = true;
    Pos pm{0, 0u};                  // input row y - 1 of the next output row
    for (int cs = lb; ok && cs < strips; cs += gk) {
      const Strip cst = strip_at(cs);
      const int x = cst.x0 + lx;
      const bool skip = x >= nx;
      Pos p0 = next(pm), pp = next(p0);
      ok = wait_full(pm) && wait_full(p0);
      for (int cr = 0; ok && cr < cst.nrows; ++cr) {
        if (!wait_full(pp)) {
          ok = false;
          break;
        }
        if (!skip) {
          const S* rows3[3] = {row_at(pm), row_at(p0), row_at(pp)};
          R h[9];
#pragma unroll
          for (int i = 0; i < 9; ++i)
            h[i] = to_r<R>(rows3[1 - cy(i)][i * Lay::W + lx + Lay::A - cx(i)]);
          const uint32_t word = reinterpret_cast<const uint32_t*>(
              reinterpret_cast<const unsigned char*>(rows3[1]) + Lay::ROW_BYTES)[lx >> 5];
          finish_node<S, COLL>(m, sc, A, B, x, cst.y0 + cr, ((word >> (lx & 31)) & 1u) != 0, t,
                               h, fx, fy, touched, bad);
        }
        release(pm);                // row y - 1 is not read again
        pm = p0;
        p0 = pp;
        pp = next(pp);
      }
      if (ok) {
        release(pm);
        release(p0);
        pm = pp;                    // the next strip's first input row
      }
    }
    if (!ok) {
      atomicOr(m.status, DEV_TIMEOUT);
      s_abort = 1;
    }
  }
  // the block's force partial: its strip's slot when partials go per strip
  // (recomputed here rather than kept live through the loop)
  const int bb = block_role(p).idx;
  const int sgb = p.strip_order ? p.strip_order[bb] : bb;
  const int slot = p.strip_force ? p.strip_force[sgb] : sgb;
  // dataflow (one strip per block: sgb is the strip's index in the table):
  // the partial slot of step t last held step t-2's partials; they must be
  // reduced (by a block of launch t-1) before they are overwritten
  if (p.strip_done && slot >= 0 && threadIdx.x == 0 &&
      !wait_at_least(p.reduced + (p.n_members == 1 ? 0 : p.strip_member[sgb]), t - 1, m.status))
    atomicOr(m.status, DEV_TIMEOUT);
  write_partial(p, t, slot, fx, fy, touched, bad, m.status);
  if (p.strip_done) {
    // every thread's stores of this strip (ordered with the copies of the
    // next step that read them), then its completion of step t
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(p.strip_done + sgb, t + 1);
    }
  }
}

// One block streams the rows of its strips (local strips lb, lb + gk, ... of
// member m) through an NS-slot ring with warp specialisation: warp 4 is the
// producer -- its lane 0 waits until a slot is released ("empty" barrier,
// one arrival per consumer warp), then stages the next row into it with
// cp.async.bulk completing on the slot's "full" barrier -- and warps 0-3 are
// consumers, each waiting on "full", colliding its 32 columns and releasing
// the slot.  No block-wide barrier per row: warps run ahead independently.
template <typename S, int COLL, int NS>
__device__ __forceinline__ void bulk_run_rows(const StepParams& p, const Member& m, int lb,
                                              int gk, unsigned char* smem) {
  using R = typename Compute<S>::R;
  using Lay = BulkLayout<S>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * Lay::STAGE_BYTES);
  uint64_t* empty = full + NS;
  __shared__ int s_abort;
  const S* A = static_cast<const S*>(m.buf[p.q]);
  S* __restrict__ B = static_cast<S*>(m.buf[1 - p.q]);
  const int plane = m.plane, pitch = m.pitch;
  const int nx = m.nx, ny = m.ny, tiles_x = m.tiles_x, rows = p.rows;
  const int strips = m.strip_count;
  const int warp = threadIdx.x >> 5;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  const int64_t t = step_index(p);
  const bool flow = p.strip_done != nullptr;   // one strip per block (variant 6)
  if (p.strip_done && threadIdx.x == kConsumerWarps * 32) {
    // the producer lane: wait for the strips around this one (and, in an east
    // tile, the boundary blocks next to it) to complete step t-1; the fence
    // orders those acquires before its bulk copies (async proxy)
    bool ok = wait_strip_neighbours(p, m, lb, t);
    const int c = lb % m.tiles_x, L = m.nx - 1;
    if (ok && m.ext_kind != 0 && (c << 7) + 127 >= L - 4) {
      const int y0 = (lb / m.tiles_x) * p.rows;
      ok = wait_east(p, m, y0 - 2, min(y0 + p.rows, m.ny) + 1, t, false, true);
    }
    if (!ok) atomicOr(m.status, DEV_TIMEOUT);
    asm volatile("fence.proxy.async.global;" ::: "memory");
  }
  __syncthreads();
  // set-up done: wait for the previous step to complete before touching the
  // populations (it may still be reading the buffer this step writes)
  if (!flow) pdl_wait();

  // strip geometry
  struct Strip {
    int y0, x0, lead, nrows;
  };
  auto strip_at = [&](int ls) {
    Strip st;
    st.y0 = (ls / tiles_x) * rows;
    st.x0 = (ls % tiles_x) << 7;
    st.lead = st.x0 == 0 ? 0 : Lay::A;
    st.nrows = min(rows, ny - st.y0);
    return st;
  };

  double fx = 0.0, fy = 0.0;
  bool touched = false, bad = false;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if ((threadIdx.x & 31) == 0) {
      int ps = lb, pr = 0, k = 0;
      Strip pst = strip_at(lb);
      while (ps < strips) {
        const int slot = k % NS;
        if (k >= NS && !mbar_wait_bounded(&empty[slot], (uint32_t)(((k / NS) - 1) & 1))) {
          atomicOr(m.status, DEV_TIMEOUT);
          s_abort = 1;
          break;
        }
        if (s_abort) break;
        const int y = pst.y0 + pr;
        unsigned char* st = smem + slot * Lay::STAGE_BYTES;
        mbar_expect_tx(&full[slot], Lay::TX_BYTES);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          int sy = y - cy(i);
          sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
          const int sx = cx(i) == 1 ? pst.x0 - pst.lead : pst.x0;
          bulk_copy_g2s(st + i * Lay::SEG_BYTES, A + i * plane + sy * pitch + sx,
                        (uint32_t)Lay::SEG_BYTES, &full[slot]);
        }
        bulk_copy_g2s(st + 9 * Lay::SEG_BYTES,
                      m.solid_bits + y * m.words_per_row + (pst.x0 >> 5), 16u, &full[slot]);
        ++k;
        if (++pr == pst.nrows) {
          pr = 0;
          ps += gk;
          if (ps < strips) pst = strip_at(ps);
        }
      }
      // no copy may land after the block exits: wait (bounded) for the last
      // item staged into each slot
      for (int kk = k > NS ? k - NS : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NS], (uint32_t)((kk / NS) & 1));
    }
  } else {
    // ---------------- consumers ----------------
    const int lx = threadIdx.x;     // column within the 128-wide tile
    const Scalars<R> sc(m);
    int cs = lb, cr = 0, j = 0;
    Strip cst = strip_at(lb);
    int x = cst.x0 + lx;
    bool west = !m.x_periodic && x == 0;
    bool east = !m.x_periodic && x == nx - 1;
    bool skip = x >= nx;
    while (cs < strips) {
      const int slot = j % NS;
      // warp-uniform outcome, so the warp never diverges around __syncwarp
      const bool ready = __all_sync(
          0xffffffffu, !s_abort && mbar_wait_bounded(&full[slot], (uint32_t)((j / NS) & 1)));
      if (!ready) {
        atomicOr(m.status, DEV_TIMEOUT);
        s_abort = 1;
        break;
      }
      const int y = cst.y0 + cr;
      const unsigned char* st = smem + slot * Lay::STAGE_BYTES;
      if (!skip) {
        const S* seg = reinterpret_cast<const S*>(st);
        R h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int idx = cx(i) == 1 ? lx - 1 + cst.lead : (cx(i) == 0 ? lx : lx + 1);
          h[i] = to_r<R>(seg[i * Lay::SEG + (idx < 0 ? 0 : idx)]);
        }
        if (x == 0 || x == nx - 1) {
          // periodic wrap of the x +- 1 neighbours at the lattice edges
          const int ym = y == 0 ? ny - 1 : y - 1;
          const int yp = y == ny - 1 ? 0 : y + 1;
          // (A is not __restrict__: these plain loads must not take the
          // non-coherent path, the previous launch may still be writing A)
          if (x == 0) {
            h[1] = to_r<R>(A[1 * plane + y * pitch + nx - 1]);
            h[5] = to_r<R>(A[5 * plane + ym * pitch + nx - 1]);
            h[8] = to_r<R>(A[8 * plane + yp * pitch + nx - 1]);
          }
          if (x == nx - 1) {
            h[3] = to_r<R>(A[3 * plane + y * pitch]);
            h[6] = to_r<R>(A[6 * plane + ym * pitch]);
            h[7] = to_r<R>(A[7 * plane + yp * pitch]);
          }
        }
        const uint32_t word =
            reinterpret_cast<const uint32_t*>(st + 9 * Lay::SEG_BYTES)[lx >> 5];
        const int o = y * pitch + x;
        // the network blocks rebuild external east fluid nodes; solid ones stay here
        if ((word >> (lx & 31)) & 1u)
          solid_node<S, R>(A, B, m, x, y, o, h, fx, fy, touched);
        else if (!(east && m.east_mode == EAST_EXTERNAL))
          fluid_node<S, R, COLL>(B, m, sc, t, west, east, y, o, h, bad);
      }
      __syncwarp();
      if ((threadIdx.x & 31) == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot]))
                     : "memory");
      ++j;
      if (++cr == cst.nrows) {
        cr = 0;
        cs += gk;
        if (cs < strips) {
          cst = strip_at(cs);
          x = cst.x0 + lx;
          west = !m.x_periodic && x == 0;
          east = !m.x_periodic && x == nx - 1;
          skip = x >= nx;
        }
      }
    }
  }
  // the block's force partial: its strip's slot when partials go per strip
  // (recomputed here rather than kept live through the loop)
  const int bb = block_role(p).idx;
  const int sgb = p.strip_order ? p.strip_order[bb] : bb;
  const int slot = p.strip_force ? p.strip_force[sgb] : sgb;
  // dataflow (one strip per block: sgb is the strip's index in the table):
  // the partial slot of step t last held step t-2's partials; they must be
  // reduced (by a block of launch t-1) before they are overwritten
  if (p.strip_done && slot >= 0 && threadIdx.x == 0 &&
      !wait_at_least(p.reduced + (p.n_members == 1 ? 0 : p.strip_member[sgb]), t - 1, m.status))
    atomicOr(m.status, DEV_TIMEOUT);
  write_partial(p, t, slot, fx, fy, touched, bad, m.status);
  if (p.strip_done) {
    // every thread's stores of this strip (ordered with the bulk copies of
    // the next step that read them), then its completion of step t
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release(p.strip_done + sgb, t + 1);
    }
  }
}

// Variants 3, 4 and 6: FP16 storage streams row windows (one tensor copy per
// input row); FP32 and FP64 storage stage each output row's nine source
// segments (their consumers are bound by DRAM and the FP64 pipe, where the
// windows' wider rows cost more than their fewer copies save).
template <typename S, int COLL, int NS>
__device__ __forceinline__ void bulk_run(const StepParams& p, const Member& m, int lb, int gk,
                                         unsigned char* smem) {
  if constexpr (sizeof(S) == 2)
    bulk_run_window<S, COLL, NS>(p, m, lb, gk, smem);
  else
    bulk_run_rows<S, COLL, NS>(p, m, lb, gk, smem);
}

// Persistent staged kernel with dynamic strip assignment (variant 5): a
// resident-sized grid whose producers take the next strip of the launch
// table from a global counter, so blocks that run faster take more strips.
// The producer records each staged row's strip and row in the slot; consumer
// warps follow it, switching member records when the strip changes.  Forces
// go to one partial per strip and consumer warp, so the fixed-order
// reduction stays independent of which block took which strip.  The last
// block to finish resets the counters for the next launch.
template <typename S, int COLL, int NS>
__device__ __forceinline__ void bulk_run_dyn(const StepParams& p, int n_blocks,
                                             unsigned char* smem) {
  using R = typename Compute<S>::R;
  using Lay = BulkLayout<S>;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NS * Lay::STAGE_BYTES);
  uint64_t* empty = full + NS;
  __shared__ int s_abort;
  __shared__ int s_strip[NS];     // global strip of the row staged in each slot (-1: none left)
  __shared__ int s_row[NS];       // row of that strip
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int strips_total = p.dyn_strips;
  unsigned long long* ctr = p.dyn_ctr;   // [0] next strip, [1] finished blocks

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  pdl_wait();
  const int64_t t = step_index(p);
  const int rows = p.rows;

  if (warp == kConsumerWarps) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int k = 0;
      // the next strip is claimed one strip ahead, so the atomic's round trip
      // overlaps the copies of the current strip
      int sg = (int)atomicAdd(ctr, 1ull);
      for (;;) {
        const int sg_next = sg >= strips_total ? sg : (int)atomicAdd(ctr, 1ull);
        const bool done = sg >= strips_total;
        if (!done && p.strip_order) sg = p.strip_order[sg];   // strips holding solids first
        const Member& m = p.members[done || p.n_members == 1 ? 0 : p.strip_member[sg]];
        const S* __restrict__ A = static_cast<const S*>(m.buf[p.q]);
        const int ls = done ? 0 : sg - m.strip_first;
        const int y0 = (ls / m.tiles_x) * rows;
        const int x0 = (ls % m.tiles_x) << 7;
        const int lead = x0 == 0 ? 0 : Lay::A;
        const int nrows = done ? 1 : min(rows, m.ny - y0);
        for (int r = 0; r < nrows; ++r) {
          const int slot = k % NS;
          if (k >= NS && !mbar_wait_bounded(&empty[slot], (uint32_t)(((k / NS) - 1) & 1))) {
            atomicOr(m.status, DEV_TIMEOUT);
            s_abort = 1;
            break;
          }
          if (s_abort) break;
          if (done) {
            // no strips left: an empty stage tells the consumers to stop
            s_strip[slot] = -1;
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[slot]))
                         : "memory");
            ++k;
            break;
          }
          s_strip[slot] = sg;
          s_row[slot] = r;
          const int y = y0 + r;
          unsigned char* st = smem + slot * Lay::STAGE_BYTES;
          mbar_expect_tx(&full[slot], Lay::TX_BYTES);
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            int sy = y - cy(i);
            sy = sy < 0 ? sy + m.ny : (sy >= m.ny ? sy - m.ny : sy);
            const int sx = cx(i) == 1 ? x0 - lead : x0;
            bulk_copy_g2s(st + i * Lay::SEG_BYTES, A + i * m.plane + sy * m.pitch + sx,
                          (uint32_t)Lay::SEG_BYTES, &full[slot]);
          }
          bulk_copy_g2s(st + 9 * Lay::SEG_BYTES, m.solid_bits + y * m.words_per_row + (x0 >> 5),
                        16u, &full[slot]);
          ++k;
        }
        if (done || s_abort) break;
        sg = sg_next;
      }
      // no copy may land after the block exits
      for (int kk = k > NS ? k - NS : 0; kk < k; ++kk)
        mbar_wait_bounded(&full[kk % NS], (uint32_t)((kk / NS) & 1));
    }
  } else {
    // ---------------- consumers ----------------
    const int lx = threadIdx.x;     // column within the 128-wide tile
    double* part = p.partials + (size_t)(t & 1) * 2 * p.partial_stride;
    double fx = 0.0, fy = 0.0;
    bool touched = false, bad = false;
    int cur = -1;
    const Member* mp = p.members;
    const S* A = nullptr;
    S* B = nullptr;
    int plane = 0, pitch = 0, nx = 0, ny = 0, y0 = 0, x = 0, lead = 0;
    bool west = false, east = false, skip = true, ext = false;
    Scalars<R> sc(p.members[0]);
    // the strip's force partial of this warp, in fixed slots
    auto flush = [&]() {
      if (cur < 0) return;
      const bool any = __any_sync(0xffffffffu, touched);
      double ax = fx, ay = fy;
      if (any) warp_sum2(ax, ay);
      const int fs = p.strip_force[cur];
      if (lane == 0 && fs >= 0) {
        const int slot = fs * kConsumerWarps + warp;
        part[2 * slot] = any ? ax : 0.0;
        part[2 * slot + 1] = any ? ay : 0.0;
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(mp->status, DEV_NONFINITE);
      fx = fy = 0.0;
      touched = bad = false;
    };
    for (int j = 0;; ++j) {
      const int slot = j % NS;
      const bool ready = __all_sync(
          0xffffffffu, !s_abort && mbar_wait_bounded(&full[slot], (uint32_t)((j / NS) & 1)));
      if (!ready) {
        atomicOr(mp->status, DEV_TIMEOUT);
        s_abort = 1;
        break;
      }
      const int sg = s_strip[slot];
      if (sg < 0) break;
      if (sg != cur) {
        flush();
        cur = sg;
        mp = p.members + (p.n_members == 1 ? 0 : p.strip_member[sg]);
        A = static_cast<const S*>(mp->buf[p.q]);
        B = static_cast<S*>(mp->buf[1 - p.q]);
        plane = mp->plane;
        pitch = mp->pitch;
        nx = mp->nx;
        ny = mp->ny;
        const int ls = sg - mp->strip_first;
        y0 = (ls / mp->tiles_x) * p.rows;
        const int x0 = (ls % mp->tiles_x) << 7;
        lead = x0 == 0 ? 0 : Lay::A;
        x = x0 + lx;
        west = !mp->x_periodic && x == 0;
        east = !mp->x_periodic && x == nx - 1;
        skip = x >= nx;
        ext = east && mp->east_mode == EAST_EXTERNAL;
        sc = Scalars<R>(*mp);
      }
      const int y = y0 + s_row[slot];
      const unsigned char* st = smem + slot * Lay::STAGE_BYTES;
      if (!skip) {
        const S* seg = reinterpret_cast<const S*>(st);
        R h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int idx = cx(i) == 1 ? lx - 1 + lead : (cx(i) == 0 ? lx : lx + 1);
          h[i] = to_r<R>(seg[i * Lay::SEG + (idx < 0 ? 0 : idx)]);
        }
        if (x == 0 || x == nx - 1) {
          // periodic wrap of the x +- 1 neighbours at the lattice edges
          const int ym = y == 0 ? ny - 1 : y - 1;
          const int yp = y == ny - 1 ? 0 : y + 1;
          if (x == 0) {
            h[1] = to_r<R>(A[1 * plane + y * pitch + nx - 1]);
            h[5] = to_r<R>(A[5 * plane + ym * pitch + nx - 1]);
            h[8] = to_r<R>(A[8 * plane + yp * pitch + nx - 1]);
          }
          if (x == nx - 1) {
            h[3] = to_r<R>(A[3 * plane + y * pitch]);
            h[6] = to_r<R>(A[6 * plane + ym * pitch]);
            h[7] = to_r<R>(A[7 * plane + yp * pitch]);
          }
        }
        const uint32_t word =
            reinterpret_cast<const uint32_t*>(st + 9 * Lay::SEG_BYTES)[lx >> 5];
        const int o = y * pitch + x;
        if ((word >> (lx & 31)) & 1u) {
          solid_node<S, R>(A, B, *mp, x, y, o, h, fx, fy, touched);
        } else if (!ext) {
          fluid_node<S, R, COLL>(B, *mp, sc, t, west, east, y, o, h, bad);
        }
      }
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[slot]))
                     : "memory");
    }
    flush();
  }
  // the last block out resets the counters for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ctr + 1, 1ull) == (unsigned long long)(n_blocks - 1)) {
      ctr[0] = 0ull;
      ctr[1] = 0ull;
      __threadfence();
    }
  }
}

template <typename S, int COLL, int NS, int MINB, bool EXT, bool DYN>
__global__ void __launch_bounds__(kBulkThreads, MINB) step_bulk_kernel(const StepParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  pdl_launch_dependents();
  const BlockRole role = block_role(p);
  if (EXT && role.kind == ROLE_BOUNDARY) {
    const int blk = role.idx;
    if (p.strip_done) {
      // dataflow: wait for the east strips and boundary blocks of step t-1
      // that meet this block's rows +- 2
      if (threadIdx.x == 0) {
        const Member& m = p.n_members == 1 ? p.m0 : p.members[p.nn_block_member[blk]];
        const int y0 = (blk - m.nn_first) * ext_rows(m);
        if (!wait_east(p, m, y0 - 2, min(y0 + ext_rows(m), m.ny) + 1, step_index(p), true,
                       true))
          atomicOr(m.status, DEV_TIMEOUT);
      }
      __syncthreads();
    } else {
      pdl_wait();
    }
    ext_dispatch<S>(p, blk, smem);
    if (p.strip_done) {
      // this block's east nodes (read next by bulk copies), then its flag
      asm volatile("fence.proxy.async.global;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release(p.strip_done + p.ext_flags + blk, step_index(p) + 1);
      }
    }
    return;
  }
  if (role.kind == ROLE_REDUCE) {
    pdl_wait();
    const int64_t t = step_index(p);
    if (p.reduce_prev && t >= 1) {
      reduce_force(p, role.idx, t - 1);
      publish_reduced(p, role.idx, t - 1);
    }
    return;
  }
  const int b = role.idx;   // stream-and-collide block
  const int nblocks = (int)gridDim.x - p.nn_blocks - p.n_members;
  // one block per strip: the strip order puts strips holding solid nodes first,
  // so their extra work overlaps the rest instead of trailing it
  const int sb = p.strip_order ? p.strip_order[b] : b;
  if (DYN) {
    bulk_run_dyn<S, COLL, NS>(p, nblocks, smem);
  } else if (p.n_members == 1) {
    // blocks part_count apart share the strips: part_count = strips gives one
    // strip per block, fewer blocks make them stream several strips each
    bulk_run<S, COLL, NS>(p, p.m0, sb, p.m0.strip_count > nblocks ? nblocks : p.m0.strip_count,
                          smem);
  } else {
    // stage this block's member record in shared memory once (coalesced),
    // instead of every thread chasing its fields in global memory
    __shared__ __align__(16) Member s_member;
    constexpr int kWords = (int)(sizeof(Member) / sizeof(uint64_t));
    static_assert(sizeof(Member) % sizeof(uint64_t) == 0, "Member must be 8-byte sized");
    if (threadIdx.x < 32) {
      const uint64_t* src =
          reinterpret_cast<const uint64_t*>(p.members + p.strip_member[sb]);
      uint64_t* dst = reinterpret_cast<uint64_t*>(&s_member);
      for (int w = threadIdx.x; w < kWords; w += 32) dst[w] = src[w];
    }
    __syncthreads();
    bulk_run<S, COLL, NS>(p, s_member, sb - s_member.blk_first, s_member.blk_count, smem);
  }
}


// Variants 0-2: the register-pipelined kernel with __launch_bounds__ minimum
// resident blocks of 128 threads per SM of 6, 8, 10.  Variant 3: the
// warp-specialised staged kernel (a ring of 4, 6 or 8 row slots for FP64, FP32
// or FP16 storage), one block per strip.
// Variant 4: the same on a resident-sized grid, each block streaming a fixed
// share of the strips through its ring.  Variant 5: the resident-sized grid
// taking strips from a global counter (dynamic balance).  Variant 6: variant 3
// ordered by per-strip completion flags instead of whole launches (dataflow
// between consecutive steps).
constexpr int kVariants = 7;
// ring slots of the staged kernel: with FP16 storage the consumers of
// variants 3, 4 and 6 hold three input rows (y - 1, y, y + 1) of an 8-slot
// ring; otherwise one staged output row of a 4-slot ring
template <typename S>
constexpr int bulk_slots() {
  return sizeof(S) == 2 ? 8 : 4;
}

template <typename S>
constexpr int prec_of() {
  return sizeof(S) == 8 ? LBM_FP64 : (sizeof(S) == 4 ? LBM_FP32 : LBM_FP16DEV);
}

// Launch with programmatic stream serialisation (dependent launch).
template <typename Kernel>
inline void launch_pdl(Kernel kernel, int grid, int threads, size_t smem, cudaStream_t s,
                       const StepParams& p) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, p);
}

// dynamic shared memory of launches with boundary blocks: the larger of the
// stream-and-collide need (ring), the network block's and the CBC block's
// The network blocks need the blob of the largest network of the launch
// (p.nn_blob_max floats) on top of their window; a launch without network or
// CBC members asks for no more than its stream-and-collide blocks need, so
// those keep their occupancy.
template <typename R>
inline size_t ext_need(const StepParams& p, int threads) {
  size_t v = 0;
  if (p.nn_blob_max > 0) {
    const size_t nn = sizeof(R) == 4 ? nn_tc_smem_bytes(p.nn_blob_max)
                                     : nn_smem_bytes<R>(threads / 32);
    v = v > nn ? v : nn;
  }
  if (p.has_cbc) v = v > cbc_smem_bytes<R>(threads) ? v : cbc_smem_bytes<R>(threads);
  return v;
}
template <typename R>
inline size_t ext_bulk_smem(const StepParams& p, size_t ring) {
  const size_t e = ext_need<R>(p, kBulkThreads);
  return ring > e ? ring : e;
}
// cap of the dynamic shared memory attribute of the kernels with boundary blocks
constexpr int kExtSmemCap = 160 * 1024;

template <typename S, int COLL, int MINB, bool EXT, bool DYN>
void launch_bulk(const StepParams& p, int blocks, cudaStream_t s) {
  // the dynamic shared memory attribute is set by the occupancy query that
  // every group runs at creation (occ_bulk), or for the network kernels at
  // their first launch
  using R = typename Compute<S>::R;
  size_t smem = step_bulk_smem(prec_of<S>(), bulk_slots<S>());
  if (EXT) smem = ext_bulk_smem<R>(p, smem);
  launch_pdl(step_bulk_kernel<S, COLL, bulk_slots<S>(), MINB, EXT, DYN>, p.nn_blocks + blocks + p.n_members,
             kBulkThreads, smem, s, p);
}

template <typename S, int COLL, bool EXT>
void launch_v(const StepParams& p, int variant, int blocks, cudaStream_t s) {
  using R = typename Compute<S>::R;
  const int g = p.nn_blocks + blocks + p.n_members;
  const size_t dyn = EXT ? ext_need<R>(p, 128) : 0;
  switch (variant) {
    case 0: launch_pdl(step_kernel<S, COLL, 6, EXT>, g, 128, dyn, s, p); break;
    case 1: launch_pdl(step_kernel<S, COLL, 8, EXT>, g, 128, dyn, s, p); break;
    case 2: launch_pdl(step_kernel<S, COLL, 10, EXT>, g, 128, dyn, s, p); break;
    case 5: launch_bulk<S, COLL, 6, EXT, true>(p, blocks, s); break;
    default: launch_bulk<S, COLL, 6, EXT, false>(p, blocks, s); break;
  }
}

template <typename S, bool EXT>
void launch_c(int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (coll == LBM_BGK) launch_v<S, 0, EXT>(p, variant, blocks, s);
  else if (coll == LBM_MRT) launch_v<S, 1, EXT>(p, variant, blocks, s);
  else launch_v<S, 2, EXT>(p, variant, blocks, s);
}

}  // namespace lbm
