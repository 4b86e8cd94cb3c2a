// Lattice engine: the kernel instantiations with Gibbs local moves (Methods, Eq. 5), compiled
// apart from the Metropolis ones so that the two build in parallel. Contextual proposals
// refill with Metropolis sweeps and are not combined with Gibbs sweeps.
#include "pt_lattice.cuh"

namespace pt {

cudaError_t configure_lattice_gibbs_kernels(int smem) {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel<1, 4, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 8, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 4, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 8, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<4, 8, false, true>, A, smem);
    return e;
}

cudaError_t launch_lattice_gibbs(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                                 size_t smem, const RunArgs& a, int flags, cudaStream_t stream) {
    if (maxW == 1 && kb4)
        lattice_kernel<1, 4, false, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 1)
        lattice_kernel<1, 8, false, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 2 && kb4)
        lattice_kernel<2, 4, false, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 2)
        lattice_kernel<2, 8, false, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else
        lattice_kernel<4, 8, false, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    return cudaGetLastError();
}

}  // namespace pt
