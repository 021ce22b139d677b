// kernels.cuh -- device-side data structures and the collision operator of the CUDA path.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "lattice.cuh"

namespace lbm {

// Device view of one block (mirrors BlockLayout plus the device mask pointer).
struct DevBlock {
    int32_t nx, ny, nz, pitch;
    int64_t plane, slab;
    int64_t offset;        // element offset of this block in the PDF arena arrays
    const uint32_t *mask;  // padded-layout cell masks (bit 31 non-fluid, bit i bounce-back) or nullptr
    int32_t xo;
    int32_t through;       // neighbours are read and written in place (see nbr)
    int32_t nbr[27];       // block covering each ghost-shell region, -1 = boundary / none
    int32_t wrap;          // bit a: across axis a the block is its own neighbour (nbr = itself)
    __host__ __device__ int64_t cell(int x, int y, int z) const
    {
        return (int64_t)(z + 1) * plane + (int64_t)(y + 1) * pitch + xo + x;
    }
};

constexpr uint32_t kMaskSolid = 1u << 31;

// Arena offset (elements from the base of the PDF array) of slot `q` of cell
// (x, y, z) + (dx, dy, dz) of block *Bp.  Inside the block, or outside with no neighbour in
// place (boundary region, or a block that keeps ghost copies): the own (ghost) cell.
// Outside with a neighbour in place: the neighbour block's cell -- along a crossed axis its
// first (+) or last (-) layer, along the other axes the same coordinate (faces of such
// neighbours match exactly); a block spanning a periodic axis alone is its own neighbour,
// which wraps the index.
__device__ __forceinline__ int64_t resolve(const DevBlock *__restrict__ blocks, const DevBlock *Bp, int x, int y,
                                           int z, int dx, int dy, int dz, int q)
{
    int sx = x + dx, sy = y + dy, sz = z + dz;
    const int rx = sx < 0 ? -1 : (sx >= Bp->nx ? 1 : 0);
    const int ry = sy < 0 ? -1 : (sy >= Bp->ny ? 1 : 0);
    const int rz = sz < 0 ? -1 : (sz >= Bp->nz ? 1 : 0);
    int nb = -1;
    if ((rx | ry | rz) != 0 && Bp->through) nb = Bp->nbr[(rx + 1) + 3 * (ry + 1) + 9 * (rz + 1)];
    if (nb < 0) return Bp->offset + (int64_t)q * Bp->slab + Bp->cell(sx, sy, sz);
    const DevBlock *N = blocks + nb;
    if (rx) sx = rx > 0 ? 0 : N->nx - 1;
    if (ry) sy = ry > 0 ? 0 : N->ny - 1;
    if (rz) sz = rz > 0 ? 0 : N->nz - 1;
    return N->offset + (int64_t)q * N->slab + N->cell(sx, sy, sz);
}

struct DevTile {
    int32_t block;
    int16_t x0, y0, z0;
    uint8_t flags;     // bit 0: some cell of the tile has a non-zero mask; bit 1: rows staged by bulk
                       // copies; bit 2: staged, two cells per thread over this row and the next
                       // tile's; bit 3: staged, the row is swept by the tile before
    uint8_t width_m1;  // tile width in cells - 1 (threads per CTA / width = tile height)
};

struct DevRun {
    int64_t src, dst;
    int32_t len, sstride, dstride, pad;
};

// Relaxation constants of the pair form of the collision (see collide below), per weight
// class c = |c_i|^2 (0 rest, 1 axis, 2 face diagonal, 3 corner).
template <class R>
struct Rates {
    R wp, wm;        // omega+, omega-
    R rest;          // 1 - omega+
    R alpha, beta;   // 1 - (omega+ + omega-)/2, (omega- - omega+)/2
    R pw[4], mw[4];  // omega+ w_c, 3 omega- w_c
    R pq[4];         // 4.5 omega+ w_c
};

// Collision constants, in the arithmetic type R of the sweep.
template <class R>
struct Coll {
    R omega_p, omega_m;    // TRT rates (SRT: equal)
    R a_p, a_m;            // 1 - omega/2 factors of the Guo source
    Rates<R> r;            // the rates in pair form
    R bw[4];               // Guo source: 3 a+ w_c (multiplies u.F)
    R fa[27], fc[27];      // Guo source per direction: 9 a+ w_i (c_i.F), 3 a- w_i (c_i.F)
    R F[3];                // body force
    R rho0;                // deviation base density of the storage (rho0 for *_DEV, else 0)
    R base[27];            // storage offset per direction (w_i rho0 for *_DEV storages, else 0)
    R mrt_d[4];            // MRT: rate minus the TRT rate of the bulk, fourth-, fifth-, sixth-order groups
    R cum[10];             // cumulant (D3Q27): rates of the shear, bulk, third-order sum, difference, xyz,
                           // fourth-order difference, sum, mixed, fifth- and sixth-order groups
    int cumulant;          // non-zero: the context's collision is the cumulant one (init kernel)
    int cum_unit;          // non-zero: every cumulant rate beyond the bulk is 1
};

// Pair-form rates for omega+ / omega- (host or device).
template <class R>
__host__ __device__ __forceinline__ Rates<R> rates_of(R wp, R wm, const R (&wc)[4])
{
    Rates<R> r;
    r.wp = wp;
    r.wm = wm;
    r.rest = R(1) - wp;
    r.alpha = R(1) - R(0.5) * (wp + wm);
    r.beta = R(0.5) * (wm - wp);
    for (int c = 0; c < 4; ++c) {
        r.pw[c] = wp * wc[c];
        r.mw[c] = R(3) * wm * wc[c];
        r.pq[c] = R(4.5) * wp * wc[c];
    }
    return r;
}

// ---------------------------------------------------------------------------------------
// Storage formats.  T is the stored type, R the arithmetic type.  The *_DEV formats store
// the deviation f_i - w_i rho0 (base[i]) in 16 bits.
// ---------------------------------------------------------------------------------------
// Load path of the two-grid source array (read-only during the sweep): 0 = read-only data
// path (ld.global.nc), 1 = evict-first streaming load (ld.global.cs).
#ifndef LBM_PULL_LOAD
#define LBM_PULL_LOAD 0
#endif

template <class T>
__device__ __forceinline__ T ld_src(const T *p)
{
#if LBM_PULL_LOAD == 1
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

template <class T>
struct Storage;

template <>
struct Storage<double> {
    using T = double;
    using R = double;
    static __device__ __forceinline__ R ld(const T *p, R) { return ld_src(p); }
    static __device__ __forceinline__ R ld_rw(const T *p, R) { return *p; }
    static __device__ __forceinline__ void st(T *p, R v, R) { __stcs(p, v); }
    static __device__ __forceinline__ void st_plain(T *p, R v, R) { *p = v; }
    // stored value as is (the deviation for *_DEV formats): conversion only
    static __device__ __forceinline__ R raw(const T *p) { return ld_src(p); }
    static __device__ __forceinline__ R raw_rw(const T *p) { return *p; }
    static __device__ __forceinline__ void st_raw(T *p, R v) { __stcs(p, v); }
    static __device__ __forceinline__ R stored(R v) { return v; }  // the value st_raw stores
};

template <>
struct Storage<float> {
    using T = float;
    using R = float;
    static __device__ __forceinline__ R ld(const T *p, R) { return ld_src(p); }
    static __device__ __forceinline__ R ld_rw(const T *p, R) { return *p; }
    static __device__ __forceinline__ void st(T *p, R v, R) { __stcs(p, v); }
    static __device__ __forceinline__ void st_plain(T *p, R v, R) { *p = v; }
    static __device__ __forceinline__ R raw(const T *p) { return ld_src(p); }
    static __device__ __forceinline__ R raw_rw(const T *p) { return *p; }
    static __device__ __forceinline__ void st_raw(T *p, R v) { __stcs(p, v); }
    static __device__ __forceinline__ R stored(R v) { return v; }
};

template <>
struct Storage<__nv_bfloat16> {
    using T = __nv_bfloat16;
    using R = float;
    static __device__ __forceinline__ R ld(const T *p, R base) { return base + __bfloat162float(ld_src(p)); }
    static __device__ __forceinline__ R ld_rw(const T *p, R base) { return base + __bfloat162float(*p); }
    static __device__ __forceinline__ void st(T *p, R v, R base) { __stcs(p, __float2bfloat16_rn(v - base)); }
    static __device__ __forceinline__ void st_plain(T *p, R v, R base) { *p = __float2bfloat16_rn(v - base); }
    static __device__ __forceinline__ R raw(const T *p) { return __bfloat162float(ld_src(p)); }
    static __device__ __forceinline__ R raw_rw(const T *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st_raw(T *p, R v) { __stcs(p, __float2bfloat16_rn(v)); }
    static __device__ __forceinline__ R stored(R v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

template <>
struct Storage<__half> {
    using T = __half;
    using R = float;
    static __device__ __forceinline__ R ld(const T *p, R base) { return base + __half2float(ld_src(p)); }
    static __device__ __forceinline__ R ld_rw(const T *p, R base) { return base + __half2float(*p); }
    static __device__ __forceinline__ void st(T *p, R v, R base) { __stcs(p, __float2half_rn(v - base)); }
    static __device__ __forceinline__ void st_plain(T *p, R v, R base) { *p = __float2half_rn(v - base); }
    static __device__ __forceinline__ R raw(const T *p) { return __half2float(ld_src(p)); }
    static __device__ __forceinline__ R raw_rw(const T *p) { return __half2float(*p); }
    static __device__ __forceinline__ void st_raw(T *p, R v) { __stcs(p, __float2half_rn(v)); }
    static __device__ __forceinline__ R stored(R v) { return __half2float(__float2half_rn(v)); }
};

// 1/x for the density of a cell (x > 0, normal): the hardware's approximate reciprocal refined
// by Newton-Raphson steps y <- y + y (1 - x y) with the residual taken by an FMA (Markstein's
// form; each step squares the relative error): two steps for FP64, one for FP32, which leaves
// the result within about one unit in the last place of 1/x.
__device__ __forceinline__ double recip(double x)
{
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
}
__device__ __forceinline__ float recip(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return fmaf(y, fmaf(-x, y, 1.0f), y);
}

// ---------------------------------------------------------------------------------------
// MRT groups (Eq. 3 with a diagonal S of one rate per group of moments).  The moment space is
// spanned by polynomials of c grouped by degree and made orthogonal, group against lower
// groups, under the weighted product <a, b> = sum_i w_i a(c_i) b(c_i): momentum; shear (5);
// bulk |c|^2 - 1; third order; fourth order; (D3Q27) fifth and sixth order.  With the even
// groups relaxed at omega+ and the odd ones at omega- the operator is TRT, so MRT is computed
// as TRT (omega+ = the shear rate, omega- = the third-order rate) plus, for each group g whose
// rate differs by d_g from its TRT rate, the term
//   -d_g P_g (f - feq + S/2),   (P_g h)_i = w_i sum_k p_k(c_i) [G_g^-1 m_g(h)]_k,
// m_g(h)_k = sum_i p_k(c_i) h_i, G_g the Gram matrix of the group's polynomials p_k.  The
// equilibrium and the Guo source are w_i times polynomials of degree <= 2, so their moments
// vanish in every group of degree >= 3; in the bulk group m(feq) = rho u.u and m(S) = 2 u.F.
// (The momentum rate drops out under Guo forcing and needs no term.)  Polynomials:
//   bulk: |c|^2 - 1, <p, p> = 2/3 (both lattices);
//   D3Q19 fourth order: q_ab = ca^2 cb^2 - (ca^2 + cb^2)/3 + cc^2/6 + 1/18 for ab = xy, xz, yz,
//     Gram matrix 7/162 on and -1/81 off the diagonal, G^-1 = 18 I + 12 J;
//   D3Q27 (h(a) = a^2 - 1/3): fourth order h(ca) h(cb) (<p,p> = 4/81) and cb cc h(ca) (2/81),
//     fifth order h(cb) h(cc) ca (4/243), sixth order h(cx) h(cy) h(cz) (8/729); orthogonal.
// ---------------------------------------------------------------------------------------
__host__ __device__ constexpr double mrt_h(int a) { return a * a - 1.0 / 3.0; }
__host__ __device__ constexpr double mrt_bulk(int x, int y, int z) { return x * x + y * y + z * z - 1.0; }
__host__ __device__ constexpr double mrt_q19(int a, int b, int c)
{
    return a * a * b * b - (a * a + b * b) / 3.0 + c * c / 6.0 + 1.0 / 18.0;
}

// Moments of the pre-collision populations in the corrected groups: even ones from the pair
// sums (and the rest population), odd ones from the pair differences.
template <int Q, class R>
struct MrtMoments {
    R mb;     // bulk
    R m4[6];  // fourth order: D3Q19 xy, xz, yz; D3Q27 h h (xy, xz, yz), then c c h (x, y, z)
    R m5[3];  // fifth order (D3Q27): x, y, z
    R m6;     // sixth order (D3Q27)
    __device__ __forceinline__ void rest(R f0)
    {
        mb = -f0;
        if (Q == 19) {
            for (int k = 0; k < 3; ++k) m4[k] = R(mrt_q19(0, 0, 0)) * f0;
        } else {
            for (int k = 0; k < 3; ++k) m4[k] = R(mrt_h(0) * mrt_h(0)) * f0;
            for (int k = 3; k < 6; ++k) m4[k] = R(0);
            for (int k = 0; k < 3; ++k) m5[k] = R(0);
            m6 = R(mrt_h(0) * mrt_h(0) * mrt_h(0)) * f0;
        }
    }
    // pair (i, opp i) with sum s and difference d; (x, y, z) = c_i
    __device__ __forceinline__ void pair(int x, int y, int z, R s, R d)
    {
        if (mrt_bulk(x, y, z) != 0.0) mb = fma(R(mrt_bulk(x, y, z)), s, mb);
        if (Q == 19) {
            m4[0] = fma(R(mrt_q19(x, y, z)), s, m4[0]);
            m4[1] = fma(R(mrt_q19(x, z, y)), s, m4[1]);
            m4[2] = fma(R(mrt_q19(y, z, x)), s, m4[2]);
        } else {
            m4[0] = fma(R(mrt_h(x) * mrt_h(y)), s, m4[0]);
            m4[1] = fma(R(mrt_h(x) * mrt_h(z)), s, m4[1]);
            m4[2] = fma(R(mrt_h(y) * mrt_h(z)), s, m4[2]);
            if (y * z != 0) m4[3] = fma(R(y * z * mrt_h(x)), s, m4[3]);
            if (x * z != 0) m4[4] = fma(R(x * z * mrt_h(y)), s, m4[4]);
            if (x * y != 0) m4[5] = fma(R(x * y * mrt_h(z)), s, m4[5]);
            if (x != 0) m5[0] = fma(R(x * mrt_h(y) * mrt_h(z)), d, m5[0]);
            if (y != 0) m5[1] = fma(R(y * mrt_h(x) * mrt_h(z)), d, m5[1]);
            if (z != 0) m5[2] = fma(R(z * mrt_h(x) * mrt_h(y)), d, m5[2]);
            m6 = fma(R(mrt_h(x) * mrt_h(y) * mrt_h(z)), s, m6);
        }
    }
};

// The corrections' coefficients: y_g = d_g G_g^-1 m_g (bulk: of m - rho u.u + u.F), and the
// correction of direction c = w [even(c) + odd(c)], even(c) = sum over the even groups of
// p_k(c) y_k, odd(c) likewise (the fifth order).
template <int Q, class R>
struct MrtCorr {
    R yb, y4[6], y5[3], y6;
    __device__ __forceinline__ MrtCorr() {}
    __device__ __forceinline__ MrtCorr(const MrtMoments<Q, R> &m, const R (&d)[4], R rho, R usq, R uF)
    {
        yb = d[0] * R(1.5) * (m.mb - rho * usq + uF);
        if (Q == 19) {
            const R t = R(12) * (m.m4[0] + m.m4[1] + m.m4[2]);
            for (int k = 0; k < 3; ++k) y4[k] = d[1] * fma(R(18), m.m4[k], t);
        } else {
            for (int k = 0; k < 3; ++k) y4[k] = d[1] * R(81.0 / 4.0) * m.m4[k];
            for (int k = 3; k < 6; ++k) y4[k] = d[1] * R(81.0 / 2.0) * m.m4[k];
            for (int k = 0; k < 3; ++k) y5[k] = d[2] * R(243.0 / 4.0) * m.m5[k];
            y6 = d[3] * R(729.0 / 8.0) * m.m6;
        }
    }
    __device__ __forceinline__ R even(int x, int y, int z, R w) const
    {
        R e = R(0);
        if (mrt_bulk(x, y, z) != 0.0) e = R(mrt_bulk(x, y, z)) * yb;
        if (Q == 19) {
            e = fma(R(mrt_q19(x, y, z)), y4[0], e);
            e = fma(R(mrt_q19(x, z, y)), y4[1], e);
            e = fma(R(mrt_q19(y, z, x)), y4[2], e);
        } else {
            e = fma(R(mrt_h(x) * mrt_h(y)), y4[0], e);
            e = fma(R(mrt_h(x) * mrt_h(z)), y4[1], e);
            e = fma(R(mrt_h(y) * mrt_h(z)), y4[2], e);
            if (y * z != 0) e = fma(R(y * z * mrt_h(x)), y4[3], e);
            if (x * z != 0) e = fma(R(x * z * mrt_h(y)), y4[4], e);
            if (x * y != 0) e = fma(R(x * y * mrt_h(z)), y4[5], e);
            e = fma(R(mrt_h(x) * mrt_h(y) * mrt_h(z)), y6, e);
        }
        return w * e;
    }
    __device__ __forceinline__ R odd(int x, int y, int z, R w) const
    {
        if (Q == 19) return R(0);
        R o = R(0);
        if (x != 0) o = fma(R(x * mrt_h(y) * mrt_h(z)), y5[0], o);
        if (y != 0) o = fma(R(y * mrt_h(x) * mrt_h(z)), y5[1], o);
        if (z != 0) o = fma(R(z * mrt_h(x) * mrt_h(y)), y5[2], o);
        return w * o;
    }
};

// ---------------------------------------------------------------------------------------
// Collision operator (Eq. 2-3 of the paper with SRT/TRT relaxation and Guo forcing), fused
// over opposite direction pairs.  TRT per pair (i, o = opp(i)), with s = f_i + f_o and
// d = f_i - f_o:
//   f*_i = f_i - w+ (s/2 - feq+) - w- (d/2 - feq-) + a+ S+ + a- S-
//   f*_o = f_o - w+ (s/2 - feq+) + w- (d/2 - feq-) + a+ S+ - a- S-
//   feq+ = w rho (1 + 4.5 (c.u)^2 - 1.5 u.u),  feq- = 3 w rho c.u,
//   S+ = w (9 (c.u)(c.F) - 3 u.F),  S- = 3 w c.F,  rho u = sum c f + F/2
// (SRT is the case w- = w+).  Collecting f_i and f_o:
//   f*_i = alpha f_i + beta f_o + P + M,   f*_o = alpha f_o + beta f_i + P - M,
//   alpha = 1 - (w+ + w-)/2,  beta = (w- - w+)/2,
//   P = w+ feq+ + a+ S+ = (4.5 w+ w rho) (c.u)^2 + (9 a+ w c.F)(c.u) + (w+ w rb - 3 a+ w u.F),
//   M = w- feq- + a- S- = (3 w- w rho)(c.u) + 3 a- w c.F,
// with rb = rho (1 - 1.5 u.u): per pair two FMAs for P (the brackets are per weight class or
// per direction), one for M, two each for f*_i and f*_o after P + M and P - M.  At w+ = w- = 0
// (alpha = 1, beta = 0, P = M = 0) the update is the identity bit for bit.  The same update
// holds for values stored as deviations v_i = f_i - w_i rho0 (rho0 = the deviation base; 0 for
// plain storage): since alpha + beta - 1 = -w+ the shift folds into P through
// rb = rho (1 - 1.5 u.u) - rho0, and rho = rho0 + sum v, rho u = sum c v + F/2 (sum w = 1,
// sum w c = 0).
// ---------------------------------------------------------------------------------------
// ACCURATE: relax the non-equilibrium parts s/2 - feq+ and d/2 - feq- first (the form of the
// first two equations), for full populations stored in FP32: the pair form adds terms of
// about 2 f that cancel, which near omega+ = 2 (tau -> 1/2) gives 2-3 times the rounding error
// of this form; the pair form takes fewer instructions per pair and is used where the
// arithmetic is FP64 (rounding far below any tolerance) or the stored values are deviations.
// MRT: add the group corrections above (rates in k.mrt_d; zero rates leave the TRT result).
// RCP: 1/rho from recip (above) instead of the IEEE division; the FP32 AA neighbour sweeps
// keep the division, with which the register allocator spills less there (measured).
template <int Q, bool FORCE, class R, bool ACCURATE = false, bool MRT = false, bool RCP = true>
__device__ __forceinline__ void collide(R (&f)[Q], const Coll<R> &k, const Rates<R> &rt, R rho0, R &rho_out,
                                        R &ux_out, R &uy_out, R &uz_out)
{
    using L = Lattice<Q>;
    // moments from the pair sums / differences
    R rho = rho0 + f[0], jx = R(0), jy = R(0), jz = R(0);
    MrtMoments<Q, R> mm;
    if (MRT) mm.rest(f[0]);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        const R si = f[i] + f[o];
        const R di = f[i] - f[o];
        if (MRT) mm.pair(L::cx(i), L::cy(i), L::cz(i), si, di);
        rho += si;
        if (L::cx(i) > 0) jx += di;
        if (L::cx(i) < 0) jx -= di;
        if (L::cy(i) > 0) jy += di;
        if (L::cy(i) < 0) jy -= di;
        if (L::cz(i) > 0) jz += di;
        if (L::cz(i) < 0) jz -= di;
    }
    R ux, uy, uz;
    const R inv = RCP ? recip(rho) : R(1) / rho;
    if (FORCE) {
        ux = (jx + R(0.5) * k.F[0]) * inv;
        uy = (jy + R(0.5) * k.F[1]) * inv;
        uz = (jz + R(0.5) * k.F[2]) * inv;
    } else {
        ux = jx * inv;
        uy = jy * inv;
        uz = jz * inv;
    }
    rho_out = rho;
    ux_out = ux;
    uy_out = uy;
    uz_out = uz;
    const R usq = ux * ux + uy * uy + uz * uz;
    const R rb = rho * (R(1) - R(1.5) * usq) - rho0;
    const R uF = FORCE ? ux * k.F[0] + uy * k.F[1] + uz * k.F[2] : R(0);
    R buF[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) buF[c] = FORCE ? k.bw[c] * uF : R(0);
    const R wp = rt.wp, wm = rt.wm;
    // MRT corrections (bulk, fourth..sixth order); the bulk term needs the pre-collision
    // velocity, hence after u
    const MrtCorr<Q, R> mc = MRT ? MrtCorr<Q, R>(mm, k.mrt_d, rho, usq, uF) : MrtCorr<Q, R>();
    {
        R f0;
        if (ACCURATE) {
            const R w0 = R(L::w(0));
            f0 = fma(-wp, fma(-w0, rb, f[0]), f[0]);  // f0 - w+ (f0 - feq0)
        } else {
            f0 = rt.rest * f[0] + rt.pw[0] * rb;
        }
        if (FORCE) f0 -= buF[0];
        if (MRT) f0 -= mc.even(0, 0, 0, R(L::w(0)));
        f[0] = f0;
    }
    // per weight class (pair form): 4.5 w+ w rho, w+ w rb - 3 a+ w u.F, 3 w- w rho
    R kq[4], p0[4], mr[4];
#pragma unroll
    for (int c = 1; c < 4; ++c) {
        kq[c] = rt.pq[c] * rho;
        p0[c] = FORCE ? fma(rt.pw[c], rb, -buF[c]) : rt.pw[c] * rb;
        mr[c] = rt.mw[c] * rho;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (L::opp(i) < i) continue;
        const int o = L::opp(i);
        const int c = L::cx(i) * L::cx(i) + L::cy(i) * L::cy(i) + L::cz(i) * L::cz(i);
        R cu = R(0);
        if (L::cx(i) > 0) cu += ux;
        if (L::cx(i) < 0) cu -= ux;
        if (L::cy(i) > 0) cu += uy;
        if (L::cy(i) < 0) cu -= uy;
        if (L::cz(i) > 0) cu += uz;
        if (L::cz(i) < 0) cu -= uz;
        if (ACCURATE) {
            const R rcu = rho * cu;
            const R fi = f[i], fo = f[o];
            const R w = R(L::w(i));
            const R ep = fma(R(0.5), fi + fo, -w * fma(R(4.5) * cu, rcu, rb));  // s/2 - feq+
            const R em = fma(R(0.5), fi - fo, -R(3) * w * rcu);                 // d/2 - feq-
            R gi = fma(-wp, ep, fma(-wm, em, fi));
            R go = fma(-wp, ep, fma(wm, em, fo));
            if (FORCE) {
                const R sp = fma(k.fa[i], cu, -buF[c]);  // a+ S+
                gi += sp + k.fc[i];
                go += sp - k.fc[i];
            }
            if (MRT) {
                const R E = mc.even(L::cx(i), L::cy(i), L::cz(i), R(L::w(i)));
                const R O = mc.odd(L::cx(i), L::cy(i), L::cz(i), R(L::w(i)));
                gi -= E + O;
                go -= E - O;
            }
            f[i] = gi;
            f[o] = go;
        } else {
            R P = FORCE ? fma(cu, fma(kq[c], cu, k.fa[i]), p0[c]) : fma(kq[c] * cu, cu, p0[c]);
            R M = FORCE ? fma(mr[c], cu, k.fc[i]) : mr[c] * cu;
            if (MRT) {
                P -= mc.even(L::cx(i), L::cy(i), L::cz(i), R(L::w(i)));
                M -= mc.odd(L::cx(i), L::cy(i), L::cz(i), R(L::w(i)));
            }
            const R fi = f[i], fo = f[o];
            f[i] = fma(rt.alpha, fi, fma(rt.beta, fo, P + M));
            f[o] = fma(rt.alpha, fo, fma(rt.beta, fi, P - M));
        }
    }
}

// Collision of full populations f (not deviations) with the context's constant rates.
template <int Q, bool FORCE, class R, bool MRT = false>
__device__ __forceinline__ void collide(R (&f)[Q], const Coll<R> &k)
{
    R rho, ux, uy, uz;
    collide<Q, FORCE, R, false, MRT>(f, k, k.r, R(0), rho, ux, uy, uz);
}

// Moments of a stored post-collision state, in FP64: rho = sum f*, j = sum c f* - F/2.
template <int Q>
__device__ __forceinline__ void moments_post(const double (&f)[Q], const double F[3], double &rho, double j[3])
{
    using L = Lattice<Q>;
    rho = 0.0;
    j[0] = j[1] = j[2] = 0.0;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        j[0] += L::cx(i) * f[i];
        j[1] += L::cy(i) * f[i];
        j[2] += L::cz(i) * f[i];
    }
    for (int a = 0; a < 3; ++a) j[a] -= 0.5 * F[a];
}

template <int Q>
__host__ __device__ constexpr int64_t dir_offset(int i, int64_t pitch, int64_t plane)
{
    return (int64_t)Lattice<Q>::cx(i) + (int64_t)Lattice<Q>::cy(i) * pitch + (int64_t)Lattice<Q>::cz(i) * plane;
}

}  // namespace lbm
