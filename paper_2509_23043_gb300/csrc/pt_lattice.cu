// Lattice engine: the kernel instantiations with Metropolis local moves, the small kernels
// (initial state, pool capture, state read and write) and the host-callable launchers. The
// engine's device code is in pt_lattice.cuh; the Gibbs instantiations are in
// pt_lattice_gibbs.cu.
#include "pt_lattice.cuh"

namespace pt {

// Random initial state (Algorithm 1, initialisation): word [wb][site]
// is output word 0 of Philox(site, 0, wb, id), i.e. bit b is walker 32 wb + b's spin.
__global__ void lattice_init_kernel(const LatInst* __restrict__ insts, uint64_t seed) {
    const LatInst& I = insts[blockIdx.x];
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = threadIdx.x; i < I.W * I.N; i += blockDim.x) {
        const int wb = i / I.N, site = i - wb * I.N;
        const uint4 r = philox(make_uint4((uint32_t)site, 0u, (kDomInit << 24) | (uint32_t)wb, I.iid),
                               k0, k1);
        I.spins[i] = r.x;
    }
}

// Copy slot configurations of a source batch into pool entry `entry` of a destination
// batch (bit strings, site order).
__global__ void lattice_capture_kernel(const LatInst* __restrict__ dst,
                                       const LatInst* __restrict__ src, int entry) {
    const LatInst& D = dst[blockIdx.x];
    const LatInst& Sr = src[blockIdx.x];
    const int N = Sr.N, NW = Sr.NW;
    for (int idx = threadIdx.x; idx < Sr.R * NW; idx += blockDim.x) {
        const int r = idx / NW, k = idx - r * NW;
        const int w = Sr.wos[r];
        const uint32_t* sp = Sr.spins + (w >> 5) * N;
        uint32_t word = 0;
        for (int b = 0; b < 32; ++b) {
            const int i = k * 32 + b;
            if (i < N) word |= ((sp[i] >> (w & 31)) & 1u) << b;
        }
        uint32_t* out = const_cast<uint32_t*>(D.pool) + (size_t)entry * D.pstride + (size_t)r * NW + k;
        *out = word;
    }
}

// Unpack the configurations of one instance in slot order into int8 [R][N].
__global__ void lattice_read_kernel(const LatInst* __restrict__ insts, int inst, int8_t* out) {
    const LatInst& I = insts[inst];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < I.R * I.N;
         idx += gridDim.x * blockDim.x) {
        const int r = idx / I.N, i = idx - r * I.N;
        const int w = I.wos[r];
        out[idx] = ((I.spins[(w >> 5) * I.N + i] >> (w & 31)) & 1u) ? 1 : -1;
    }
}

// Write one instance's configurations (int8 [R][N], slot order) with walker ids per slot.
__global__ void lattice_write_kernel(const LatInst* __restrict__ insts, int inst,
                                     const int8_t* in, const int32_t* walker) {
    const LatInst& I = insts[inst];
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < I.W * I.N;
         idx += gridDim.x * blockDim.x) {
        const int wb = idx / I.N, i = idx - wb * I.N;
        uint32_t word = 0;
        for (int r = 0; r < I.R; ++r) {
            const int w = walker[r];
            if ((w >> 5) == wb && in[(size_t)r * I.N + i] > 0) word |= 1u << (w & 31);
        }
        I.spins[idx] = word;
    }
}

// ------------------------------------------------------------------------------------
// host-callable launchers
// ------------------------------------------------------------------------------------
// Defined in pt_lattice_gibbs.cu: the same for the Gibbs instantiations.
cudaError_t configure_lattice_gibbs_kernels(int smem);
cudaError_t launch_lattice_gibbs(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                                 size_t smem, const RunArgs& a, int flags, cudaStream_t stream);

// Defined in pt_lattice_big.cu: the instantiations with the spins in global memory.
cudaError_t configure_lattice_gsp_kernels(int smem);
cudaError_t launch_lattice_gsp(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                               size_t smem, const RunArgs& a, int flags, cudaStream_t stream);

// The kernels' dynamic shared-memory limit is raised once, outside any stream capture.
cudaError_t configure_lattice_kernels(int smem) {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(lattice_kernel<1, 4, false, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 8, false, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 4, false, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 8, false, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<4, 8, false, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 4, true, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<1, 8, true, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 4, true, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<2, 8, true, false>, A, smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lattice_kernel<4, 8, true, false>, A, smem);
    if (e == cudaSuccess) e = configure_lattice_gibbs_kernels(smem);
    if (e == cudaSuccess) e = configure_lattice_gsp_kernels(smem);
    return e;
}

// kb4: the group's counts fit in 4 bits (at most two words per thread per colour class).
template <bool CTX>
cudaError_t launch_lattice_t(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                             size_t smem, const RunArgs& a, int flags, cudaStream_t stream) {
    if (maxW == 1 && kb4)
        lattice_kernel<1, 4, CTX, false><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 1)
        lattice_kernel<1, 8, CTX, false><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 2 && kb4)
        lattice_kernel<2, 4, CTX, false><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else if (maxW == 2)
        lattice_kernel<2, 8, CTX, false><<<n, threads, smem, stream>>>(d_insts, a, flags);
    else
        lattice_kernel<4, 8, CTX, false><<<n, threads, smem, stream>>>(d_insts, a, flags);
    return cudaGetLastError();
}

cudaError_t launch_lattice(const LatInst* d_insts, int n, int maxW, int kb4, int threads,
                           size_t smem, const RunArgs& a, int flags, cudaStream_t stream) {
    if (flags & kGlobalSpins)
        return launch_lattice_gsp(d_insts, n, maxW, kb4, threads, smem, a, flags, stream);
    if (flags & kGibbs)
        return launch_lattice_gibbs(d_insts, n, maxW, kb4, threads, smem, a, flags, stream);
    if (flags & kWithContext)
        return launch_lattice_t<true>(d_insts, n, maxW, kb4, threads, smem, a, flags, stream);
    return launch_lattice_t<false>(d_insts, n, maxW, kb4, threads, smem, a, flags, stream);
}

cudaError_t launch_lattice_init(const LatInst* d, int n, uint64_t seed, cudaStream_t s) {
    lattice_init_kernel<<<n, 256, 0, s>>>(d, seed);
    return cudaGetLastError();
}
cudaError_t launch_lattice_capture(const LatInst* dst, const LatInst* src, int n, int entry,
                                   cudaStream_t s) {
    lattice_capture_kernel<<<n, 256, 0, s>>>(dst, src, entry);
    return cudaGetLastError();
}
cudaError_t launch_lattice_read(const LatInst* d, int inst, int8_t* out, int total, cudaStream_t s) {
    lattice_read_kernel<<<(total + 255) / 256, 256, 0, s>>>(d, inst, out);
    return cudaGetLastError();
}
cudaError_t launch_lattice_write(const LatInst* d, int inst, const int8_t* in, const int32_t* walker,
                                 int total, cudaStream_t s) {
    lattice_write_kernel<<<(total + 255) / 256, 256, 0, s>>>(d, inst, in, walker);
    return cudaGetLastError();
}

}  // namespace pt
