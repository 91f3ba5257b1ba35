// The step kernels with fused boundary blocks for the east column (NN direct
// reconstruction, Sec. 3.1, Eq. 15; characteristic outflow, Sec. 4, Eqs.
// 17-28): the same templates as step.cu, instantiated with the boundary
// dispatch compiled in, in a translation unit of their own so that launches
// with the Zou & He outflow run kernels without that code.
#include "step_kernels.cuh"

namespace lbm {

namespace {

template <typename S, int COLL>
void set_bulk_smem_attr() {
  static bool done = false;
  if (done) return;
  // a cap: each launch passes what its members need (ext_need)
  const int cap = kExtSmemCap;
  cudaFuncSetAttribute(step_bulk_kernel<S, COLL, bulk_slots<S>(), 6, true, false>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(step_bulk_kernel<S, COLL, bulk_slots<S>(), 6, true, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(step_kernel<S, COLL, 6, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(step_kernel<S, COLL, 8, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  cudaFuncSetAttribute(step_kernel<S, COLL, 10, true>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
  done = true;
}

template <typename S>
void launch_nn_c(int coll, const StepParams& p, int variant, int blocks, cudaStream_t s) {
  if (coll == LBM_BGK) set_bulk_smem_attr<S, 0>();
  else if (coll == LBM_MRT) set_bulk_smem_attr<S, 1>();
  else set_bulk_smem_attr<S, 2>();
  launch_c<S, true>(coll, p, variant, blocks, s);
}

}  // namespace

void launch_step_ext(int prec, int coll, const StepParams& p, int variant, int blocks,
                     cudaStream_t s) {
  if (prec == LBM_FP64) launch_nn_c<double>(coll, p, variant, blocks, s);
  else if (prec == LBM_FP32) launch_nn_c<float>(coll, p, variant, blocks, s);
  else launch_nn_c<__half>(coll, p, variant, blocks, s);
}

}  // namespace lbm
