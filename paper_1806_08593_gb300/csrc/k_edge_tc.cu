// k_edge_tc.cu -- tcgen05 tensor-core edge kernels (not built yet: reports unsupported).
#include "tmc_tc.cuh"

namespace tmc {
namespace tc {

tmc_status supported(const std::vector<NodeInfo>&, int) { return TMC_ERR_UNSUPPORTED; }
void workspace_layout(TcWork&, const std::vector<NodeInfo>&, long long, long long, std::vector<TcSub>&) {}
tmc_status prepare(TcWork&, const std::vector<NodeInfo>&, const std::vector<Tile>&, int, int) {
  return TMC_ERR_UNSUPPORTED;
}
void release(TcWork&) {}
void launch_pack(TcWork&, const Dev&, cudaStream_t) {}
void launch_edge_fwd(TcWork&, const Dev&, int, cudaStream_t) {}
void launch_edge_bwd(TcWork&, const Dev&, int, cudaStream_t) {}
void launch_unpack_grads(TcWork&, const Dev&, cudaStream_t) {}

}  // namespace tc
}  // namespace tmc
