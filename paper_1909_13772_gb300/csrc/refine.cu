// refine.cu -- the transfers of a static 2:1 grid refinement between a coarse and a fine
// context (Sec. 5.1.1: non-uniform grids by the mass-conserving method of Rohde et al.).
// The host builds, once, one entry per ghost slot that a sweep reads across a refinement
// face (api.cu, lbm_refine_create):
//   explosion (into the fine context's ghost slots, before each of its two steps): the coarse
//     post-collision population of the coarse cell that holds the fine ghost cell the value
//     streams from -- one fine cell away for the first fine step, two for the second;
//   coalescence (into the coarse context's ghost slots, after the first fine step): the mean
//     over the 8 fine cells inside the coarse cell of the populations that leave the fine grid
//     into it during the two fine steps, 4 emitted at the start of the second fine step (the
//     state after the first) and 4 at the start of the first (the state before it).
// One thread per entry; the element size is that of the storage format.
#include "launch.hpp"

namespace lbm {

namespace {

template <class T>
__global__ void __launch_bounds__(256) k_explode(T *__restrict__ dst, const T *__restrict__ src,
                                                 const int64_t *__restrict__ ent, int64_t n, int sub)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    dst[ent[3 * k]] = src[ent[3 * k + sub]];
}

template <class T>
__global__ void __launch_bounds__(256) k_coalesce(T *__restrict__ dst, const T *__restrict__ fnew,
                                                  const T *__restrict__ fhalf, const int64_t *__restrict__ ent,
                                                  int64_t n)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t *e = ent + 9 * k;
    T s = T(0);
#pragma unroll
    for (int j = 1; j <= 4; ++j) s += fnew[e[j]];
#pragma unroll
    for (int j = 5; j <= 8; ++j) s += fhalf[e[j]];
    dst[e[0]] = s * T(0.125);
}

template <class T>
cudaError_t explode(const RefineArgs &a)
{
    const int64_t ctas = (a.n + 255) / 256;
    if (ctas > 0x7fffffffLL || (a.sub != 1 && a.sub != 2)) return cudaErrorInvalidValue;
    k_explode<T><<<(unsigned)ctas, 256, 0, a.stream>>>((T *)a.dst, (const T *)a.src, a.ent, a.n, a.sub);
    return cudaGetLastError();
}

template <class T>
cudaError_t coalesce(const RefineArgs &a)
{
    const int64_t ctas = (a.n + 255) / 256;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_coalesce<T><<<(unsigned)ctas, 256, 0, a.stream>>>((T *)a.dst, (const T *)a.src, (const T *)a.src2, a.ent, a.n);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine_explode(const RefineArgs &a)
{
    if (a.n <= 0) return cudaSuccess;
    if (a.elem_bytes == 8) return explode<double>(a);
    if (a.elem_bytes == 4) return explode<float>(a);
    return cudaErrorInvalidValue;
}

cudaError_t launch_refine_coalesce(const RefineArgs &a)
{
    if (a.n <= 0) return cudaSuccess;
    if (a.elem_bytes == 8) return coalesce<double>(a);
    if (a.elem_bytes == 4) return coalesce<float>(a);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
