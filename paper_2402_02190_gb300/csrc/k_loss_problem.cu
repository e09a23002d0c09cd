// The fused loss kernels (loss_impl.cuh) instantiated for one problem.  The
// build compiles this file once per problem with -DCPRA_LOSS_PROBLEM=<p>
// (0 MIS, 1 MaxCut, 2 DBM, 3 weighted MIS, 4 MaxCut with edge weights), so
// that the five sets of instances -- every row width, G in FP32 and BF16 --
// compile in parallel; k_loss.cu dispatches to them.
#include "loss_impl.cuh"

#ifndef CPRA_LOSS_PROBLEM
#error "k_loss_problem.cu is compiled with -DCPRA_LOSS_PROBLEM=<problem>"
#endif

namespace cpra {

template <>
int loss_launch_problem<CPRA_LOSS_PROBLEM>(const LossArgs& a, int nch, int max_grid,
                                           int staged_grid, cudaStream_t st) {
  if (a.dg == DT_BF16)
    return dispatch_loss<CPRA_LOSS_PROBLEM, bf16, true>(a, nch, max_grid, staged_grid, st);
  return dispatch_loss<CPRA_LOSS_PROBLEM, float, true>(a, nch, max_grid, staged_grid, st);
}

#if CPRA_LOSS_PROBLEM == 0
int loss_launch_bits(const LossArgs& a, int nch, int max_grid, cudaStream_t st) {
  return dispatch_loss<0, float, false>(a, nch, max_grid, max_grid, st);
}
#endif

#ifdef CPRA_CHECKED
template <>
void csr_check_collect_loss<CPRA_LOSS_PROBLEM>(CsrCheck* r) {
  CPRA_CSR_CHECK_COLLECT(r);
}
#endif

}  // namespace cpra
