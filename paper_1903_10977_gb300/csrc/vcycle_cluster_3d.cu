// 3-D instances of the cluster-resident coarse V-cycle.
#include "vcycle_cluster.cuh"

namespace imgm {

const void* ds_kernel_3d(int p) {
    return p == 1 ? (const void*)k_vcycle_dsmem<3, 1>
         : p == 2 ? (const void*)k_vcycle_dsmem<3, 2>
         : p == 3 ? (const void*)k_vcycle_dsmem<3, 3> : nullptr;
}

}  // namespace imgm
