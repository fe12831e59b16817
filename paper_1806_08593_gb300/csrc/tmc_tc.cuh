// tmc_tc.cuh -- tensor-core (tcgen05) path: workspace, packing and launchers.
#pragma once
#include <vector>

#include "../../include/tmc.h"
#include "tmc_internal.cuh"

namespace tmc {
namespace tc {

struct TcSub {
  void** dst;
  size_t bytes;
};

struct TcWork {
  int precision = 0;
};

tmc_status supported(const std::vector<NodeInfo>& nodes, int precision);
void workspace_layout(TcWork& w, const std::vector<NodeInfo>& nodes, long long nk, long long nkd,
                      std::vector<TcSub>& subs);
tmc_status prepare(TcWork& w, const std::vector<NodeInfo>& nodes, const std::vector<Tile>& tiles,
                   int maxK, int maxd);
void release(TcWork& w);
void launch_pack(TcWork& w, const Dev& D, cudaStream_t s);
void launch_edge_fwd(TcWork& w, const Dev& D, int level, cudaStream_t s);
void launch_edge_bwd(TcWork& w, const Dev& D, int level, cudaStream_t s);
void launch_unpack_grads(TcWork& w, const Dev& D, cudaStream_t s);

}  // namespace tc
}  // namespace tmc
