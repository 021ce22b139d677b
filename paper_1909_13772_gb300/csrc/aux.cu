// aux.cu -- boundary/ghost fill, initialisation, state import/export, macroscopic output and
// deterministic reductions.  Compiled once per (stencil, storage) pair like sweep.cu.
//
// Storage layouts of the post-collision state f*_i(x) (x a fluid interior cell):
//   LAYOUT_PULL (two-grid source array):  a[i][x]
//   LAYOUT_AA_E (after an AA local sweep): a[opp i][x]
//   LAYOUT_AA_O (after an AA neighbour sweep): a[i][x + c_i]
#include "cumulant.cuh"
#include "select.cuh"

namespace lbm {
namespace {

constexpr int kQ = LBM_Q;
using S = Storage<StoreT>;
using R = typename S::R;
using Lq = Lattice<kQ>;

// Arena offset (from the base of the PDF array) of the slot holding f*_i of cell (x, y, z)
// of block Bp in each layout.  In the AA O layout the value sits at the cell x + c_i, which
// may lie in a neighbour block read in place (resolve); a value whose target x + c_i is
// no-slip sits in the cell's own slot opp(i) (the neighbour sweep's bounce-back; m = the
// cell's mask).
__device__ __forceinline__ int64_t slot(int layout, int i, int64_t cell, const DevBlock *__restrict__ blocks,
                                        const DevBlock *Bp, int x, int y, int z, uint32_t m)
{
    if (layout == LAYOUT_PULL) return Bp->offset + (int64_t)i * Bp->slab + cell;
    if (layout == LAYOUT_AA_E) return Bp->offset + (int64_t)Lq::opp(i) * Bp->slab + cell;
    if (i > 0 && ((m >> Lq::opp(i)) & 1u)) return Bp->offset + (int64_t)Lq::opp(i) * Bp->slab + cell;
    return resolve(blocks, Bp, x, y, z, Lq::cx(i), Lq::cy(i), Lq::cz(i), i);
}

__device__ __forceinline__ uint32_t mask_of(const DevBlock &B, int64_t cell) { return B.mask ? B.mask[cell] : 0u; }

// Interior coordinates of a cell index of the padded layout.
__device__ __forceinline__ void coords_of(int64_t cell, const DevBlock &B, int &x, int &y, int &z)
{
    z = (int)(cell / B.plane) - 1;
    const int64_t r = cell - (int64_t)(z + 1) * B.plane;
    y = (int)(r / B.pitch) - 1;
    x = (int)(r - (int64_t)(y + 1) * B.pitch) - B.xo;
}

// ---------------------------------------------------------------------------------------
// Boundary links and ghost copies (one launch; Sec. 4.4 boundary lists, Sec. 3.3 local
// ghost transfer).  For a link (x, q) the outgoing post-collision PDF v = f*_q(x) hits the
// boundary halfway to x + c_q and comes back as the incoming f_opp(q)(x, t+1):
//   no-slip  : v
//   velocity : v - 6 w_q rho_w (c_q . u_w)
//   pressure : -v + 2 w_q rho_w [1 + 4.5 (c_q . u_b)^2 - 1.5 u_b^2],  u_b = u(x, t)
// The result goes where the next sweep reads direction opp(q) of x:
//   pull: a[opp q][x + c_q];  AA (before neighbour sweep): a[q][x + c_q];
//   AA (before local sweep): a[opp q][x].
// Ghost runs copy the slots the next sweep reads (pull, AA forward) from the interior
// image cell to the ghost, or (AA reverse) the slots the neighbour sweep wrote into a ghost
// back to the image cell.
// ---------------------------------------------------------------------------------------
struct FillConst {
    R F[3];
    R base[27];
    double base64[27];  // the deviation base in FP64 (host-facing reads and writes)
};

// A stored PDF as f_i in FP64 (the deviation base of the *_DEV storages added in FP64), and the
// store of f_i given in FP64: the kernels that move PDFs to and from the host and the FP64
// reductions use these, so that no FP32 rounding of w_i rho0 + v_i enters them.
__device__ __forceinline__ double ld_f64(const StoreT *p, const FillConst &k, int i)
{
    return (double)S::raw_rw(p) + k.base64[i];
}
__device__ __forceinline__ void st_f64(StoreT *p, double v, const FillConst &k, int i)
{
    S::st_raw(p, R(v - k.base64[i]));
}

template <int MODE>
__global__ void __launch_bounds__(256) k_fill(StoreT *__restrict__ A, const DevBlock *__restrict__ blocks,
                                              const uint64_t *__restrict__ links, int64_t nlinks,
                                              const DevRun *__restrict__ runs, int64_t nruns, int64_t link_ctas,
                                              const double *__restrict__ params, FillConst k)
{
    if ((int64_t)blockIdx.x < link_ctas) {
        const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (l >= nlinks) return;
        const uint64_t w = links[l];
        const int q = (int)(w & 31u);
        const int kind = (int)((w >> 5) & 3u);
        const int bits = (int)((w >> 7) & 7u);
        const int par = (int)((w >> 10) & 255u);
        const int blk = (int)((w >> 18) & 0x3fffu);
        const int64_t cell = (int64_t)(w >> 32);
        const DevBlock *Bp = blocks + blk;
        const DevBlock &B = *Bp;
        const int o = Lq::opp(q);
        int cx0, cy0, cz0;
        coords_of(cell, B, cx0, cy0, cz0);
        // slots of the boundary cell x + c_q: own ghost / solid cell, or a neighbour block's cell
        int64_t src, dst;
        int layout;
        if (MODE == FILL_PULL) {
            src = B.offset + (int64_t)q * B.slab + cell;
            dst = resolve(blocks, Bp, cx0, cy0, cz0, Lq::cx(q), Lq::cy(q), Lq::cz(q), o);
            layout = LAYOUT_PULL;
        } else if (MODE == FILL_AA_E) {
            src = B.offset + (int64_t)o * B.slab + cell;
            dst = resolve(blocks, Bp, cx0, cy0, cz0, Lq::cx(q), Lq::cy(q), Lq::cz(q), q);
            layout = LAYOUT_AA_E;
        } else {
            src = resolve(blocks, Bp, cx0, cy0, cz0, Lq::cx(q), Lq::cy(q), Lq::cz(q), q);
            dst = B.offset + (int64_t)o * B.slab + cell;
            layout = LAYOUT_AA_O;
        }
        const R v = S::ld_rw(A + src, k.base[q]);
        const R wq = R(Lq::w(q));
        const R cx = R(Lq::cx(q)), cy = R(Lq::cy(q)), cz = R(Lq::cz(q));
        R out;
        if (kind == 1) {
            out = v;
        } else if (kind == 2) {
            const double *p = params + 4 * par;
            const R cu = cx * R(p[0]) + cy * R(p[1]) + cz * R(p[2]);
            out = v - R(6) * wq * R(p[3]) * cu;
        } else {
            const double *p = params + 4 * par;
            const uint32_t m0 = mask_of(B, cell);
            R rho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                const R fi = S::ld_rw(A + slot(layout, i, cell, blocks, Bp, cx0, cy0, cz0, m0), k.base[i]);
                rho += fi;
                jx += R(Lq::cx(i)) * fi;
                jy += R(Lq::cy(i)) * fi;
                jz += R(Lq::cz(i)) * fi;
            }
            const R inv = R(1) / rho;
            const R ux = (jx - R(0.5) * k.F[0]) * inv, uy = (jy - R(0.5) * k.F[1]) * inv,
                    uz = (jz - R(0.5) * k.F[2]) * inv;
            const R cu = cx * ux + cy * uy + cz * uz;
            const R usq = ux * ux + uy * uy + uz * uz;
            out = -v + R(2) * wq * R(p[3]) * (R(1) + R(4.5) * cu * cu - R(1.5) * usq);
        }
        S::st_plain(A + dst, out, k.base[o]);
    } else {
        const int64_t gt = ((int64_t)blockIdx.x - link_ctas) * blockDim.x + threadIdx.x;
        const int64_t r = gt >> 5;
        const int lane = threadIdx.x & 31;
        if (r >= nruns) return;
        const DevRun run = runs[r];
        for (int e = lane; e < run.len; e += 32) {
            const int64_t s = run.src + (int64_t)e * run.sstride;
            const int64_t d = run.dst + (int64_t)e * run.dstride;
            if (MODE == FILL_AA_O)
                A[s] = A[d];
            else
                A[d] = A[s];
        }
    }
}

// ---------------------------------------------------------------------------------------
// Wet-node (Zou-He) velocity and pressure faces, two-grid pull layout, D3Q19 (Sec. 5.1.1
// names the in- and outflow family; Zou & He 1997, Hecht & Harting 2010 for D3Q19).  Run after
// the fill, before the sweep: for a node x (fluid cell of the first layer at the face, inward
// normal n) the populations the pull sweep will gather are known for c.n <= 0 (read where the
// sweep reads them: the neighbour's slot, or the cell's own opposite slot where a no-slip bit
// bounces); with K0 (c.n = 0) and Km (c.n < 0) their sums and j = rho u - F/2,
//   velocity face: rho = (K0 + 2 Km - F.n/2) / (1 - u_w.n), j = rho u_w - F/2;
//   pressure face: rho = rho_w, j.n = rho_w - K0 - 2 Km, j.t = -F.t/2;
// the unknown c.n > 0 ones are f_c = f_-c + j.n/3 (c = n) and f_-c + (j.n + s j.t)/6 - s N_t
// (c = n + s t), N_t = (1/2) sum_{c.n = 0} (c.t) f - j.t/3, written into the ghost slot the sweep
// pulls them from.  One thread per node.
// ---------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_zouhe(StoreT *__restrict__ A, const DevBlock *__restrict__ blocks,
                                               const uint64_t *__restrict__ nodes, int64_t nnodes,
                                               const double *__restrict__ params, int pressure_faces, FillConst k)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnodes || kQ != 19) return;
    const uint64_t w = nodes[t];
    const int face = (int)(w & 7u), a = face / 2;
    const int nrm = (face & 1) ? -1 : 1;  // inward normal along axis a
    const int blk = (int)((w >> 3) & 0x3fffu);
    const int64_t cell = (int64_t)(w >> 32);
    const DevBlock *Bp = blocks + blk;
    const DevBlock &B = *Bp;
    int x, y, z;
    coords_of(cell, B, x, y, z);
    const uint32_t m = mask_of(B, cell);
    R f[kQ];
    R K0 = R(0), Km = R(0), T[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int c3[3] = {Lq::cx(i), Lq::cy(i), Lq::cz(i)};
        const int cn = c3[a] * nrm;
        if (cn > 0) continue;
        const int64_t src = (i > 0 && ((m >> i) & 1u)) ? B.offset + (int64_t)Lq::opp(i) * B.slab + cell
                                                      : resolve(blocks, Bp, x, y, z, -c3[0], -c3[1], -c3[2], i);
        f[i] = S::ld_rw(A + src, k.base[i]);
        if (cn == 0) {
            K0 += f[i];
            T[0] += R(c3[0]) * f[i];
            T[1] += R(c3[1]) * f[i];
            T[2] += R(c3[2]) * f[i];
        } else {
            Km += f[i];
        }
    }
    const double *p = params + 4 * face;
    R rho, j[3];
    if ((pressure_faces >> face) & 1) {
        rho = R(p[3]);
        for (int b = 0; b < 3; ++b) j[b] = -R(0.5) * k.F[b];
        j[a] = (rho - K0 - R(2) * Km) * R(nrm);
    } else {
        rho = (K0 + R(2) * Km - R(0.5) * k.F[a] * R(nrm)) / (R(1) - R(p[a]) * R(nrm));
        for (int b = 0; b < 3; ++b) j[b] = rho * R(p[b]) - R(0.5) * k.F[b];
    }
    const R jn = j[a] * R(nrm);
    const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int c3[3] = {Lq::cx(i), Lq::cy(i), Lq::cz(i)};
        if (c3[a] * nrm <= 0) continue;
        const R fo = f[Lq::opp(i)];
        R v = fo + jn / R(3);
        const int tt = c3[t1] != 0 ? t1 : (c3[t2] != 0 ? t2 : -1);
        if (tt >= 0) {
            const R s = R(c3[tt]);
            const R Nt = R(0.5) * T[tt] - j[tt] / R(3);
            v = fo + (jn + s * j[tt]) / R(6) - s * Nt;
        }
        S::st_plain(A + resolve(blocks, Bp, x, y, z, -c3[0], -c3[1], -c3[2], i), v, k.base[i]);
    }
}

// ---------------------------------------------------------------------------------------
// Per-cell kernels over one block's interior (thread per cell, n = x + nx (y + ny z)).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t cell_of(int64_t n, const DevBlock &B, int &x, int &y, int &z)
{
    x = (int)(n % B.nx);
    const int64_t t = n / B.nx;
    y = (int)(t % B.ny);
    z = (int)(t / B.ny);
    return (int64_t)(z + 1) * B.plane + (int64_t)(y + 1) * B.pitch + B.xo + x;
}

// The context's collision of full populations: the cumulant one for D3Q27 contexts that use
// it, else SRT/TRT/MRT (the MRT terms vanish unless the context is MRT).
template <bool FORCE, int Q>
__device__ __forceinline__ void init_collide(R (&f)[Q], const Coll<R> &k)
{
    if constexpr (Q == 27) {
        if (k.cumulant) {
            R rho, ux, uy, uz;
            collide_cumulant<FORCE, true>(f, k, rho, ux, uy, uz);
            return;
        }
    }
    collide<Q, FORCE, R, true>(f, k);
}

// Initial state: populations = equilibrium at (rho, u - F/(2 rho)), then one collision
// (the stored state is post-collision).  Equilibrium: w rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u).
template <bool FORCE>
__global__ void k_init(StoreT *__restrict__ A, const DevBlock *__restrict__ blocks, int blk, int layout,
                       const double *__restrict__ rho_in, const double *__restrict__ u_in,
                       const uint32_t *__restrict__ mask, Coll<R> k)
{
    const DevBlock *Bp = blocks + blk;
    const DevBlock &B = *Bp;
    const int64_t N = (int64_t)B.nx * B.ny * B.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int x, y, z;
    const int64_t cell = cell_of(n, B, x, y, z);
    StoreT *a = A + B.offset;
    const uint32_t m = mask ? mask[cell] : 0u;
    if (m & kMaskSolid) return;  // non-fluid cells hold no state
    const R rho = R(rho_in[n]);
    R ux = R(u_in[n]), uy = R(u_in[N + n]), uz = R(u_in[2 * N + n]);
    if (FORCE) {
        ux -= R(0.5) * k.F[0] / rho;
        uy -= R(0.5) * k.F[1] / rho;
        uz -= R(0.5) * k.F[2] / rho;
    }
    const R usq = ux * ux + uy * uy + uz * uz;
    R f[kQ];
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const R cu = R(Lq::cx(i)) * ux + R(Lq::cy(i)) * uy + R(Lq::cz(i)) * uz;
        f[i] = R(Lq::w(i)) * rho * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
    }
    init_collide<FORCE>(f, k);
#pragma unroll
    for (int i = 0; i < kQ; ++i) S::st_plain(A + slot(layout, i, cell, blocks, Bp, x, y, z, m), f[i], k.base[i]);
}

// PDFs of the box [r0, r0 + rn) of the block's interior cells, out[i * N + n], n = x + rx (y + ry z)
// relative to the box (the whole block: r0 = 0, rn = its size).
__global__ void k_get(const StoreT *__restrict__ A, const DevBlock *__restrict__ blocks, int blk, int layout,
                      double *__restrict__ out, const uint32_t *__restrict__ mask, FillConst k, int3 r0, int3 rn)
{
    const DevBlock *Bp = blocks + blk;
    const DevBlock &B = *Bp;
    const int64_t N = (int64_t)rn.x * rn.y * rn.z;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int x = r0.x + (int)(n % rn.x);
    const int y = r0.y + (int)((n / rn.x) % rn.y);
    const int z = r0.z + (int)(n / ((int64_t)rn.x * rn.y));
    const int64_t cell = B.cell(x, y, z);
    const StoreT *a = A + B.offset;
    const uint32_t m = mask ? mask[cell] : 0u;
    const bool fluid = !(m & kMaskSolid);
    for (int i = 0; i < kQ; ++i)
        out[(int64_t)i * N + n] = fluid ? ld_f64(A + slot(layout, i, cell, blocks, Bp, x, y, z, m), k, i) : 0.0;
}

__global__ void k_set(StoreT *__restrict__ A, const DevBlock *__restrict__ blocks, int blk, int layout,
                      const double *__restrict__ in,
                      const uint32_t *__restrict__ mask, FillConst k)
{
    const DevBlock *Bp = blocks + blk;
    const DevBlock &B = *Bp;
    const int64_t N = (int64_t)B.nx * B.ny * B.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int x, y, z;
    const int64_t cell = cell_of(n, B, x, y, z);
    const uint32_t m = mask ? mask[cell] : 0u;
    if (m & kMaskSolid) return;
    StoreT *a = A + B.offset;
    for (int i = 0; i < kQ; ++i)
        st_f64(A + slot(layout, i, cell, blocks, Bp, x, y, z, m), in[(int64_t)i * N + n], k, i);
}

// Output moments in FP64: rho = sum f*, u = (sum c f* - F/2) / rho.
__global__ void k_macro(const StoreT *__restrict__ A, const DevBlock *__restrict__ blocks, int blk, int layout,
                        double *__restrict__ rho_out,
                        double *__restrict__ u_out, const uint32_t *__restrict__ mask, FillConst k, double Fx,
                        double Fy, double Fz)
{
    const DevBlock *Bp = blocks + blk;
    const DevBlock &B = *Bp;
    const int64_t N = (int64_t)B.nx * B.ny * B.nz;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int x, y, z;
    const int64_t cell = cell_of(n, B, x, y, z);
    const uint32_t m = mask ? mask[cell] : 0u;
    if (m & kMaskSolid) {
        rho_out[n] = 0.0;
        u_out[n] = u_out[N + n] = u_out[2 * N + n] = 0.0;
        return;
    }
    // Sums as accurate as FP64 ones at a fraction of their cost (GB300's FP64 rate is 1/64 of
    // its FP32 rate): FP32 storage sums its values as float-float pairs (TwoSum, Knuth: s = a + b,
    // b' = s - a, e = (a - (s - b')) + (b - b') gives a + b = s + e exactly), converted to FP64
    // once; the other storages sum in FP64 (the 16-bit ones add their deviation base there).
    // No products with c_i in {-1, 0, 1}, one division.
    double rho, jx, jy, jz;
    if (LBM_ST == 1) {
        float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
        auto add = [&](int a, float v) {
            const float t = h[a] + v, bp = t - h[a];
            l[a] += (h[a] - (t - bp)) + (v - bp);
            h[a] = t;
        };
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const float fi = (float)S::raw_rw(A + slot(layout, i, cell, blocks, Bp, x, y, z, m));
            add(0, fi);
            if (Lq::cx(i) != 0) add(1, Lq::cx(i) > 0 ? fi : -fi);
            if (Lq::cy(i) != 0) add(2, Lq::cy(i) > 0 ? fi : -fi);
            if (Lq::cz(i) != 0) add(3, Lq::cz(i) > 0 ? fi : -fi);
        }
        rho = (double)h[0] + (double)l[0];
        jx = (double)h[1] + (double)l[1];
        jy = (double)h[2] + (double)l[2];
        jz = (double)h[3] + (double)l[3];
    } else {
        rho = jx = jy = jz = 0.0;
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const StoreT *p = A + slot(layout, i, cell, blocks, Bp, x, y, z, m);
            const double fi = LBM_ST >= 2 ? ld_f64(p, k, i) : (double)S::raw_rw(p);
            rho += fi;
            if (Lq::cx(i) > 0) jx += fi;
            if (Lq::cx(i) < 0) jx -= fi;
            if (Lq::cy(i) > 0) jy += fi;
            if (Lq::cy(i) < 0) jy -= fi;
            if (Lq::cz(i) > 0) jz += fi;
            if (Lq::cz(i) < 0) jz -= fi;
        }
    }
    jx = fma(-0.5, Fx, jx);
    jy = fma(-0.5, Fy, jy);
    jz = fma(-0.5, Fz, jz);
    const double inv = 1.0 / rho;
    rho_out[n] = rho;
    u_out[n] = jx * inv;
    u_out[N + n] = jy * inv;
    u_out[2 * N + n] = jz * inv;
}

// Box sums for coarse-graining: one thread per coarse cell of r^3 interior cells; sums over
// its fluid cells of rho, rho u (3) and rho u_a u_b (xx, yy, zz, xy, xz, yz), with u as in
// k_macro.  out[m * Nc + c], c = X + NX (Y + NY Z).
__global__ void __launch_bounds__(256) k_coarse(const StoreT *__restrict__ A, const DevBlock *__restrict__ blocks,
                                                int blk, int layout, int r, double *__restrict__ out,
                                                const uint32_t *__restrict__ mask, FillConst k, double Fx, double Fy,
                                                double Fz)
{
    const DevBlock *Bp = blocks + blk;
    const DevBlock &B = *Bp;
    const int NX = B.nx / r, NY = B.ny / r, NZ = B.nz / r;
    const int64_t Nc = (int64_t)NX * NY * NZ;
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= Nc) return;
    const int X = (int)(c % NX);
    const int Y = (int)((c / NX) % NY);
    const int Z = (int)(c / ((int64_t)NX * NY));
    const double F[3] = {Fx, Fy, Fz};
    double acc[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int dz = 0; dz < r; ++dz)
        for (int dy = 0; dy < r; ++dy)
            for (int dx = 0; dx < r; ++dx) {
                const int x = X * r + dx, y = Y * r + dy, z = Z * r + dz;
                const int64_t cell = (int64_t)(z + 1) * B.plane + (int64_t)(y + 1) * B.pitch + B.xo + x;
                const uint32_t m = mask ? mask[cell] : 0u;
                if (m & kMaskSolid) continue;
                double f[kQ];
#pragma unroll
                for (int i = 0; i < kQ; ++i)
                    f[i] = ld_f64(A + slot(layout, i, cell, blocks, Bp, x, y, z, m), k, i);
                double rho, j[3];
                moments_post<kQ>(f, F, rho, j);
                const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
                acc[0] += rho;
                acc[1] += rho * u[0];
                acc[2] += rho * u[1];
                acc[3] += rho * u[2];
                acc[4] += rho * u[0] * u[0];
                acc[5] += rho * u[1] * u[1];
                acc[6] += rho * u[2] * u[2];
                acc[7] += rho * u[0] * u[1];
                acc[8] += rho * u[0] * u[2];
                acc[9] += rho * u[1] * u[2];
            }
#pragma unroll
    for (int q = 0; q < 10; ++q) out[(int64_t)q * Nc + c] = acc[q];
}

// ---------------------------------------------------------------------------------------
// Deterministic FP64 reduction over all fluid cells: per tile (CTA) partial sums reduced by
// warp shuffles, then a fixed-order sum of the partials (diag.cu, launch_reduce_final).
// Partial record: mass, j_x, j_y, j_z, kinetic energy, max |u|, non-finite cells, fluid cells.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void __launch_bounds__(256) k_reduce_tiles(const StoreT *__restrict__ A, const DevBlock *__restrict__ blocks,
                                                      const DevTile *__restrict__ tiles, int tx, int tz, int layout,
                                                      FillConst k, double Fx, double Fy, double Fz,
                                                      double *__restrict__ partials)
{
    const DevTile t = tiles[blockIdx.x];
    const DevBlock *Bp = blocks + t.block;
    const DevBlock &B = *Bp;
    const int ttx = (int)t.width_m1 + 1;
    const int rows = blockDim.x / ttx;  // the tile's height; leftover threads stay idle
    const int lx = threadIdx.x % ttx, ly = threadIdx.x / ttx;
    const int x = t.x0 + lx, y = t.y0 + ly;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const double F[3] = {Fx, Fy, Fz};
    if (ly < rows && x < B.nx && y < B.ny) {
        const int zend = min((int)t.z0 + tz, B.nz);
        const StoreT *a = A + B.offset;
        for (int z = t.z0; z < zend; ++z) {
            const int64_t cell = (int64_t)(z + 1) * B.plane + (int64_t)(y + 1) * B.pitch + B.xo + x;
            const uint32_t m = mask_of(B, cell);
            if (m & kMaskSolid) continue;
            double f[kQ];
            bool finite = true;
#pragma unroll
            for (int i = 0; i < kQ; ++i) {
                f[i] = ld_f64(A + slot(layout, i, cell, blocks, Bp, x, y, z, m), k, i);
                finite = finite && isfinite(f[i]);
            }
            double rho, j[3];
            moments_post<kQ>(f, F, rho, j);
            const double j2 = j[0] * j[0] + j[1] * j[1] + j[2] * j[2];
            acc[0] += rho;
            acc[1] += j[0];
            acc[2] += j[1];
            acc[3] += j[2];
            acc[4] += 0.5 * j2 / rho;
            acc[5] = fmax(acc[5], sqrt(j2) / rho);
            acc[6] += finite ? 0.0 : 1.0;
            acc[7] += 1.0;
        }
    }
    __shared__ double sh[8][8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const double v = c == 5 ? warp_max(acc[c]) : warp_sum(acc[c]);
        if (lane == 0) sh[warp][c] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        const int c = threadIdx.x;
        double v = 0.0;
        for (int w2 = 0; w2 < nwarps; ++w2) v = c == 5 ? fmax(v, sh[w2][c]) : v + sh[w2][c];
        partials[(int64_t)blockIdx.x * 8 + c] = v;
    }
}


FillConst fill_const(const double F[3], const double base[27])
{
    FillConst k;
    for (int a = 0; a < 3; ++a) k.F[a] = (R)F[a];
    for (int i = 0; i < 27; ++i) {
        k.base[i] = (R)base[i];
        k.base64[i] = base[i];
    }
    return k;
}

template <int MODE>
cudaError_t go_fill(const FillArgs &s)
{
    const int threads = 256;
    const int64_t link_ctas = (s.nlinks + threads - 1) / threads;
    const int64_t run_ctas = (s.nruns * 32 + threads - 1) / threads;
    const int64_t ctas = link_ctas + run_ctas;
    if (ctas == 0) return cudaSuccess;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_fill<MODE><<<(unsigned)ctas, threads, 0, s.stream>>>((StoreT *)s.a, s.blocks, s.links, s.nlinks, s.runs, s.nruns,
                                                         link_ctas, s.params, fill_const(s.F, s.base));
    return cudaGetLastError();
}

}  // namespace

cudaError_t LBM_CAT(launch_fill_, LBM_Q, LBM_ST)(const FillArgs &s)
{
    switch (s.mode) {
        case FILL_PULL: return go_fill<FILL_PULL>(s);
        case FILL_AA_E: return go_fill<FILL_AA_E>(s);
        case FILL_AA_O: return go_fill<FILL_AA_O>(s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t LBM_CAT(launch_zouhe_, LBM_Q, LBM_ST)(const FillArgs &s)
{
    if (s.nzouhe <= 0) return cudaSuccess;
    if (LBM_Q != 19) return cudaErrorInvalidValue;
    const int64_t ctas = (s.nzouhe + 255) / 256;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_zouhe<<<(unsigned)ctas, 256, 0, s.stream>>>((StoreT *)s.a, s.blocks, s.zouhe, s.nzouhe, s.params,
                                                  s.zouhe_pressure, fill_const(s.F, s.base));
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_cells_, LBM_Q, LBM_ST)(int op, int force, const CellArgs &s)
{
    const int64_t N = (int64_t)s.blk.nx * s.blk.ny * s.blk.nz;
    if (N == 0) return cudaSuccess;
    const int threads = 256;
    const int64_t ctas = (N + threads - 1) / threads;
    if (ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
    const FillConst fk = fill_const(s.F, s.base);
    const Coll<R> &k = coll_of(s.cd, s.cf, (R *)nullptr);
    switch (op) {
        case CELL_INIT:
            if (force)
                k_init<true><<<(unsigned)ctas, threads, 0, s.stream>>>((StoreT *)s.a, s.blocks, s.block, s.layout, s.rho, s.u, s.mask, k);
            else
                k_init<false><<<(unsigned)ctas, threads, 0, s.stream>>>((StoreT *)s.a, s.blocks, s.block, s.layout, s.rho, s.u, s.mask, k);
            break;
        case CELL_GET: {
            // region (the whole block when rn is zero)
            const int3 r0 = s.rn[0] ? make_int3(s.r0[0], s.r0[1], s.r0[2]) : make_int3(0, 0, 0);
            const int3 rn = s.rn[0] ? make_int3(s.rn[0], s.rn[1], s.rn[2]) : make_int3(s.blk.nx, s.blk.ny, s.blk.nz);
            const int64_t Nr = (int64_t)rn.x * rn.y * rn.z;
            k_get<<<(unsigned)((Nr + threads - 1) / threads), threads, 0, s.stream>>>(
                (const StoreT *)s.a, s.blocks, s.block, s.layout, s.f64, s.mask, fk, r0, rn);
            break;
        }
        case CELL_SET:
            k_set<<<(unsigned)ctas, threads, 0, s.stream>>>((StoreT *)s.a, s.blocks, s.block, s.layout, s.f64, s.mask, fk);
            break;
        case CELL_COARSE: {
            const int r = s.ratio;
            if (r < 1 || s.blk.nx % r || s.blk.ny % r || s.blk.nz % r) return cudaErrorInvalidValue;
            const int64_t Nc = N / ((int64_t)r * r * r);
            k_coarse<<<(unsigned)((Nc + threads - 1) / threads), threads, 0, s.stream>>>(
                (const StoreT *)s.a, s.blocks, s.block, s.layout, r, s.f64, s.mask, fk, s.F[0], s.F[1], s.F[2]);
            break;
        }
        case CELL_MACRO:
            k_macro<<<(unsigned)ctas, threads, 0, s.stream>>>((const StoreT *)s.a, s.blocks, s.block, s.layout, s.rho, s.u, s.mask,
                                                              fk, s.F[0], s.F[1], s.F[2]);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t LBM_CAT(launch_reduce_, LBM_Q, LBM_ST)(const ReduceArgs &s)
{
    if (s.ntiles <= 0 || s.ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (s.tx * s.ty > 256) return cudaErrorInvalidConfiguration;
    const FillConst fk = fill_const(s.F, s.base);
    k_reduce_tiles<<<(unsigned)s.ntiles, s.tx * s.ty, 0, s.stream>>>((const StoreT *)s.a, s.blocks, s.tiles, s.tx, s.tz,
                                                                    s.layout, fk, s.F[0], s.F[1], s.F[2], s.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_final(s.partials, s.ntiles, s.out, s.stream);
}

}  // namespace lbm
