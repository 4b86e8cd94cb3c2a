// Lattice engine: the instantiations for instances whose spins and neighbour table do not fit
// shared memory (L up to 20 with R up to 128). Their {word, complement} spins live in a
// global working copy and the table is read in place (both L2-resident); the thresholds,
// energies, labels and staging stay in shared memory. Compiled apart so that the shared-memory
// instantiations build in parallel. Contextual proposals are not combined with them.
#include "pt_lattice.cuh"

namespace pt {

cudaError_t configure_lattice_gsp_kernels(int smem) {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel<1, 4, false, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 8, false, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 4, false, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 8, false, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<4, 8, false, false, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 4, false, true, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 8, false, true, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 4, false, true, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 8, false, true, true>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<4, 8, false, true, true>, A, smem);
    return e;
}

template <bool GIBBS>
cudaError_t launch_lattice_gsp_t(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                                 size_t smem, const RunArgs& a, int flags, cudaStream_t stream) {
    if (maxW == 1 && kb4)
        lattice_kernel<1, 4, false, GIBBS, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 1)
        lattice_kernel<1, 8, false, GIBBS, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 2 && kb4)
        lattice_kernel<2, 4, false, GIBBS, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 2)
        lattice_kernel<2, 8, false, GIBBS, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else
        lattice_kernel<4, 8, false, GIBBS, true><<<n, threads, smem, stream>>>(d_insts, a, flags);
    return cudaGetLastError();
}

cudaError_t launch_lattice_gsp(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                               size_t smem, const RunArgs& a, int flags, cudaStream_t stream) {
    if (flags & kGibbs) return launch_lattice_gsp_t<true>(d_insts, n, maxW, kb4, threads, smem, a, flags, stream);
    return launch_lattice_gsp_t<false>(d_insts, n, maxW, kb4, threads, smem, a, flags, stream);
}

}  // namespace pt
