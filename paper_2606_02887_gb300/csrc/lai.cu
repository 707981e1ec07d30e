// LAI-SNMPBB operator (Sec. 2.3).  Sketch construction and the U (E (U^T X)) product.
#include "lai.cuh"

namespace snmf {

int lai_apply(const LaiOp&, int, const Dims&, const void*, void*, double, const void*, const void*,
              const void*, double*, const int*, cudaStream_t) {
  return 0;
}

int lai_build(LaiOp&, const AxArgs&, int, int64_t, int, int, int, uint64_t, int, cudaStream_t,
              std::string& msg) {
  msg = "LAI sketch not built";
  return -2;
}

void lai_free(LaiOp& op) {
  cudaFree(op.U); cudaFree(op.lam); cudaFree(op.xpart); cudaFree(op.M);
  op = LaiOp{};
}

}  // namespace snmf
