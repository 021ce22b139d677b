// halo.cu -- pack and unpack of the ghost-layer halo of a partitioned run (Sec. 3.3: only the
// PDFs that cross into a neighbour's ghost layer are exchanged, packed into one buffer per
// neighbour rank).  The copies are plain element moves between a context's PDF array and a
// caller-owned device buffer along precomputed runs (plan.hpp HaloRun); the element size is
// that of the storage format.
#include "launch.hpp"

namespace lbm {

namespace {

// One warp per run: element e of run r moves between arena[r.arena + e * r.astride] and
// buf[r.buf + e] (to_buf: arena -> buffer).
template <class T>
__global__ void __launch_bounds__(256) k_halo(T *__restrict__ arena, T *__restrict__ buf, const HaloDevRun *__restrict__ runs,
                                              int64_t nruns, int to_buf)
{
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nruns) return;
    const HaloDevRun run = runs[r];
    for (int e = lane; e < run.len; e += 32) {
        const int64_t a = run.arena + (int64_t)e * run.astride;
        if (to_buf)
            buf[run.buf + e] = arena[a];
        else
            arena[a] = buf[run.buf + e];
    }
}

template <class T>
cudaError_t go(const HaloArgs &h)
{
    const int64_t ctas = (h.nruns * 32 + 255) / 256;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_halo<T><<<(unsigned)ctas, 256, 0, h.stream>>>((T *)h.arena, (T *)h.buf, h.runs, h.nruns, h.to_buf);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_halo(const HaloArgs &h)
{
    if (h.nruns <= 0) return cudaSuccess;
    switch (h.elem_bytes) {
        case 8: return go<unsigned long long>(h);
        case 4: return go<unsigned int>(h);
        case 2: return go<unsigned short>(h);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
