// 2-D instances of the cluster-resident coarse V-cycle, and its host side: the cluster size
// this device admits, and the launch.
#include "vcycle_cluster.cuh"

namespace imgm {

const void* ds_kernel_2d(int p) {
    return p == 1 ? (const void*)k_vcycle_dsmem<2, 1>
         : p == 2 ? (const void*)k_vcycle_dsmem<2, 2>
         : p == 3 ? (const void*)k_vcycle_dsmem<2, 3> : nullptr;
}

int ds_cluster_size() {
    static int cs = -1;
    if (cs < 0) {
        cs = 0;
        const void* kerns[] = {ds_kernel_2d(1), ds_kernel_2d(2), ds_kernel_2d(3),
                               ds_kernel_3d(1), ds_kernel_3d(2), ds_kernel_3d(3)};
        for (const void* k : kerns) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) cudaGetLastError();
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DS_SMEM_MAX) != cudaSuccess)
                cudaGetLastError();
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16, 1, 1);
        cfg.blockDim = dim3(DS_TPB, 1, 1);
        cfg.dynamicSmemBytes = DS_SMEM_MAX;
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeClusterDimension;
        attr.val.clusterDim.x = 16;
        attr.val.clusterDim.y = 1;
        attr.val.clusterDim.z = 1;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxPotentialClusterSize(&n, ds_kernel_2d(2), &cfg) == cudaSuccess && n > 0)
            cs = n >= 16 ? 16 : (n >= 8 ? 8 : 0);
        else
            cudaGetLastError();
    }
    return cs;
}

cudaError_t launch_vcycle_dsmem(int dim, int p, const DsVcycle& V, cudaStream_t s) {
    if (V.cs <= 0 || V.cs != ds_cluster_size() || V.smem_bytes > DS_SMEM_MAX) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(V.cs, 1, 1);
    cfg.blockDim = dim3(DS_TPB, 1, 1);
    cfg.dynamicSmemBytes = V.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = V.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_allowed(s) ? 2 : 1;
    ++t_launches;
    const void* k = dim == 2 ? ds_kernel_2d(p) : dim == 3 ? ds_kernel_3d(p) : nullptr;
    if (k == nullptr) return cudaErrorInvalidValue;
    void* args[] = {const_cast<DsVcycle*>(&V)};
    return cudaLaunchKernelExC(&cfg, k, args);
}

}  // namespace imgm
