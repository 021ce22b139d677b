// sweep_sparse.cu -- the two-grid sweep over a fluid-cell list (porous geometries).
//
// Compiled once per (stencil, storage) pair like sweep.cu; defines launch_sparse_<Q>_<ST>.
//
// A dense block stores every cell; on a sphere packing most rows mix solid and fluid cells,
// so the dense sweep reads sectors that are partly solid and runs warps with idle lanes.  The
// fluid-cell list (plan.hpp SparsePlan) stores only fluid cells, numbered block by block in
// (z, y, x) order, each direction's values contiguous: a warp sweeps 32 consecutive fluid
// cells, writes 32 consecutive entries per direction and reads, per direction, the entries
// its table nbr names -- consecutive too wherever the neighbouring row is fluid as well.
// The method is the same (Eq. 2, pull form, fused stream and collide, Sec. 5.1.2): for fluid
// cell n and direction i the population streaming in is src[i][nbr_i(n)] (a fluid cell of
// this or a neighbour block, or the slot a boundary link filled), or for a no-slip source the
// halfway bounce-back src[opp i][n]; then the same collision as the dense sweep.  Every cell
// does the dense sweep's arithmetic, so the two layouts give the same bits.
// Algorithmic bytes per fluid-cell update: 2 Q s of PDFs plus 4 (Q - 1) of table.
#include "cell.cuh"

namespace lbm {

namespace {

template <bool FORCE, bool DIAG>
__global__ void __launch_bounds__(256, 4)
    k_sparse_sweep(const StoreT *__restrict__ src, StoreT *__restrict__ dst, const int32_t *__restrict__ nbr,
                   int64_t nfluid, int64_t stride, Coll<R> k, double *__restrict__ partials)
{
    using L = Lattice<kQ>;
    Diag<DIAG> dg;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n < nfluid) {
        R f[kQ];
        f[0] = S::raw(src + n);
#pragma unroll
        for (int i = 1; i < kQ; ++i) {
            const int32_t v = __ldg(nbr + (int64_t)(i - 1) * nfluid + n);
            const int64_t e = v == kListBounce ? (int64_t)L::opp(i) * stride + n : (int64_t)i * stride + v;
            f[i] = S::raw(src + e);
        }
        R rho, ux, uy, uz;
        collide<kQ, FORCE, R, kAccurate>(f, k, k.r, k.rho0, rho, ux, uy, uz);
        dg.add(f, k.rho0, rho, ux, uy, uz);
#pragma unroll
        for (int i = 0; i < kQ; ++i) S::st_raw(dst + (int64_t)i * stride + n, f[i]);
    }
    dg.tile_record(partials);
}

// Boundary links of the list layout: link k of fluid cell n along q (velocity or pressure)
// writes entry nfluid + k of direction opp(q), which the next sweep reads as direction opp(q) of n
// (the dense fill's arithmetic, aux.cu).
__global__ void __launch_bounds__(256) k_sparse_fill(StoreT *__restrict__ A, const uint64_t *__restrict__ links,
                                                     int64_t nlinks, int64_t nfluid, int64_t stride,
                                                     const double *__restrict__ params, Coll<R> k)
{
    using Lq = Lattice<kQ>;
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlinks) return;
    const uint64_t w = links[l];
    const int q = (int)(w & 31u);
    const int kind = (int)((w >> 5) & 3u);
    const int par = (int)((w >> 10) & 255u);
    const int64_t n = (int64_t)(w >> 32);
    const int o = Lq::opp(q);
    const R v = S::ld_rw(A + (int64_t)q * stride + n, k.base[q]);
    const R wq = R(Lq::w(q));
    const R cx = R(Lq::cx(q)), cy = R(Lq::cy(q)), cz = R(Lq::cz(q));
    const double *p = params + 4 * par;
    R out;
    if (kind == 2) {
        const R cu = cx * R(p[0]) + cy * R(p[1]) + cz * R(p[2]);
        out = v - R(6) * wq * R(p[3]) * cu;
    } else {
        R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const R fi = S::ld_rw(A + (int64_t)i * stride + n, k.base[i]);
            rho += fi;
            jx += R(Lq::cx(i)) * fi;
            jy += R(Lq::cy(i)) * fi;
            jz += R(Lq::cz(i)) * fi;
        }
        const R inv = R(1) / rho;
        const R ux = (jx - R(0.5) * k.F[0]) * inv, uy = (jy - R(0.5) * k.F[1]) * inv, uz = (jz - R(0.5) * k.F[2]) * inv;
        const R cu = cx * ux + cy * uy + cz * uz;
        const R usq = ux * ux + uy * uy + uz * uz;
        out = -v + R(2) * wq * R(p[3]) * (R(1) + R(4.5) * cu * cu - R(1.5) * usq);
    }
    S::st_plain(A + (int64_t)o * stride + nfluid + l, out, k.base[o]);
}

// Dense <-> list copies of the stored values (every direction of every fluid cell).
__global__ void __launch_bounds__(256) k_sparse_copy(StoreT *__restrict__ dense, StoreT *__restrict__ list,
                                                     const DevBlock *__restrict__ blocks,
                                                     const int32_t *__restrict__ block_of,
                                                     const int64_t *__restrict__ cell_of, int64_t nfluid, int64_t stride,
                                                     int to_list)
{
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nfluid) return;
    const DevBlock &B = blocks[block_of[n]];
    const int64_t base = B.offset + cell_of[n];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        if (to_list)
            list[(int64_t)i * stride + n] = dense[base + (int64_t)i * B.slab];
        else
            dense[base + (int64_t)i * B.slab] = list[(int64_t)i * stride + n];
    }
}

template <bool FORCE>
cudaError_t sweep(const SparseArgs &s, const Coll<R> &k)
{
    const int64_t ctas = (s.nfluid + 255) / 256;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (s.partials)
        k_sparse_sweep<FORCE, true><<<(unsigned)ctas, 256, 0, s.stream>>>((const StoreT *)s.src, (StoreT *)s.dst,
                                                                         s.nbr, s.nfluid, s.stride, k, s.partials);
    else
        k_sparse_sweep<FORCE, false><<<(unsigned)ctas, 256, 0, s.stream>>>((const StoreT *)s.src, (StoreT *)s.dst,
                                                                          s.nbr, s.nfluid, s.stride, k, nullptr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t LBM_CAT(launch_sparse_, LBM_Q, LBM_ST)(const SparseArgs &s)
{
    const Coll<R> &k = coll_of(s.cd, s.cf, (R *)nullptr);
    if (s.op == SPARSE_SWEEP) {
        if (s.nfluid <= 0) return cudaSuccess;
        return s.force ? sweep<true>(s, k) : sweep<false>(s, k);
    }
    if (s.op == SPARSE_FILL) {
        if (s.nlinks <= 0) return cudaSuccess;
        const int64_t ctas = (s.nlinks + 255) / 256;
        if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
        k_sparse_fill<<<(unsigned)ctas, 256, 0, s.stream>>>((StoreT *)s.dst, s.links, s.nlinks, s.nfluid, s.stride,
                                                           s.params, k);
        return cudaGetLastError();
    }
    if (s.nfluid <= 0) return cudaSuccess;
    const int64_t ctas = (s.nfluid + 255) / 256;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_sparse_copy<<<(unsigned)ctas, 256, 0, s.stream>>>((StoreT *)s.dense, (StoreT *)s.list, s.blocks, s.block_of,
                                                       s.cell_of, s.nfluid, s.stride, s.op == SPARSE_TO_LIST ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace lbm
