// cumulant.cuh -- the D3Q27 cumulant collision (Sec. 5.1.1: cumulants, not moments, relaxed
// towards their equilibria; Geier et al. 2015).  Included by the sweep objects built with
// -DLBM_CUMULANT_SWEEP=1 and by the init kernel.
//
// The 27 velocities are {-1,0,1}^3, so every transform between populations and moments is a
// product of one 3-point transform per axis, applied along x, y and z lines of the 3x3x3
// array g (slot (cx+1) + 3 (cy+1) + 9 (cz+1)):
//   raw moments:     (p-, p0, p+) -> (p- + p0 + p+, p+ - p-, p+ + p-)
//   central shift:   (m0, m1, m2) -> (m0, m1 - u m0, m2 - 2 u m1 + u^2 m0)
// and back.  The arithmetic runs on deviations: v_i = f_i - r0 t_i with the D3Q27 weights
// t_i = t(cx) t(cy) t(cz), t = (1/6, 2/3, 1/6) (r0 = 1 for full populations, the storage's
// rho0 for deviation storage).  The raw moments of t are W_a W_b W_c with W = (1, 0, 1/3),
// which are also the central moments of the equilibrium (the product of three 1-D
// distributions of variance 1/3), so after each central shift along an axis the part of t
// that the shift changes, r0 W W D(u) with D = (0, -u, u^2), is added explicitly; what the
// transform then yields is the excess central moment k^_abc = kappa_abc - rho W_a W_b W_c,
// zero at equilibrium.  Cumulants, their relaxation and the way back are written in these
// excess quantities, so no step subtracts two numbers near 1/3 or 1/9: FP32 keeps the
// relative accuracy of the non-equilibrium parts.
//   Density-scaled cumulants (C = rho k) of order 4..6 in excess form, with
//   a, b, c = k^_200, k^_020, k^_002 (the second-order excess) and the lower cumulants:
//     C_2pq-type: C_{2e_d+e_p+e_q} = k^ - k^_{pq}/3 - (k^_dd k^_{pq} + 2 k^_{dp} k^_{dq}) / rho
//     C_220-type: C = k^ - (k^_pp + k^_qq)/3 - (k^_pp k^_qq + 2 k^_pq^2) / rho
//     C_122-type: C = k^ - (k^_{s,2q} + k^_{s,2p})/3 - (k^_pp k^_{s,2q} + k^_qq k^_{s,2p}
//                     + 2 k^_sp k^_{p,2q} + 2 k^_sq k^_{2p,q} + 4 k^_pq k^_111) / rho
//     C_222 = k^_222 - (sum of the 4th-order diagonal pairs)/3 - (a C_022 + b C_202 + c C_220)/rho
//             - 4 (C_110 C_112 + C_101 C_121 + C_011 C_211)/rho
//             - (2 (C_210 C_012 + C_201 C_021 + C_120 C_102) + 4 C_111^2)/rho
//             - (a + b + c)/9 - (ab + bc + ca)/(3 rho) - abc/rho^2
//             - (2/3)(C_011^2 + C_101^2 + C_110^2)/rho - 2 (a C_011^2 + b C_101^2 + c C_110^2)/rho^2
//             - 8 C_110 C_101 C_011 / rho^2
//   (the moment of a product of six variables as the sum over its set partitions of the
//   products of cumulants, with the equilibrium parts rho/3, rho/9, rho/27 cancelled by hand).
//   Relaxation groups: shear (omega+; C_110, C_101, C_011, a - b, a - c), bulk (a + b + c),
//   third-order sums and differences of the pairs (C_120, C_102), (C_210, C_012), (C_201,
//   C_021), C_111, the fourth-order differences C_220 - 2 C_202 + C_022 and C_220 + C_202 -
//   2 C_022, their sum, C_211-type, fifth, sixth order -- every combination x -> x - w x.
//   A body force enters by the half-force shift of u: the first central moments are -F/2
//   before the collision and +F/2 after it.
#pragma once

#include "kernels.cuh"

namespace lbm {

__host__ __device__ constexpr int cum_slot(int i)
{
    return (Lattice<27>::cx(i) + 1) + 3 * (Lattice<27>::cy(i) + 1) + 9 * (Lattice<27>::cz(i) + 1);
}
__host__ __device__ constexpr int cix(int a, int b, int c) { return a + 3 * b + 9 * c; }

// one 3-point transform along the axis with stride ST of every line of g
template <int ST, class R, class OP>
__device__ __forceinline__ void cum_lines(R (&g)[27], OP op)
{
#pragma unroll
    for (int k = 0; k < 27; ++k) {
        if ((k / ST) % 3 != 0) continue;
        op(g[k], g[k + ST], g[k + 2 * ST], k);
    }
}

// W_a for a = the moment order along an axis (1, 0, 1/3)
__host__ __device__ constexpr double cum_w(int a) { return a == 0 ? 1.0 : (a == 1 ? 0.0 : 1.0 / 3.0); }

// central shift along AXIS of every line of g (forward: raw -> central about u, then the
// equilibrium part r0 W W D(u) added; back: that part removed, then central -> raw)
template <int AXIS, bool BACK, class R>
__device__ __forceinline__ void cum_shift(R (&g)[27], R u, R r0)
{
    constexpr int st = AXIS == 0 ? 1 : (AXIS == 1 ? 3 : 9);
    const R u2 = u * u;
#pragma unroll
    for (int k = 0; k < 27; ++k) {
        if ((k / st) % 3 != 0) continue;
        R &m0 = g[k], &m1 = g[k + st], &m2 = g[k + 2 * st];
        // the orders of the line along the two other axes
        const int a1 = AXIS == 0 ? (k / 3) % 3 : k % 3;
        const int a2 = AXIS == 2 ? (k / 3) % 3 : k / 9;
        const double ww = cum_w(a1) * cum_w(a2);
        if (!BACK) {
            m2 = fma(u2, m0, fma(R(-2) * u, m1, m2));
            m1 = fma(-u, m0, m1);
            if (ww != 0.0) {
                m1 = fma(-R(ww) * r0, u, m1);
                m2 = fma(R(ww) * r0, u2, m2);
            }
        } else {
            if (ww != 0.0) {
                m1 = fma(R(ww) * r0, u, m1);
                m2 = fma(-R(ww) * r0, u2, m2);
            }
            m2 = fma(u2, m0, fma(R(2) * u, m1, m2));
            m1 = fma(u, m0, m1);
        }
    }
}

// the second-order excess of axis d: index of k^_dd
__host__ __device__ constexpr int cdd(int d) { return d == 0 ? cix(2, 0, 0) : (d == 1 ? cix(0, 2, 0) : cix(0, 0, 2)); }
__host__ __device__ constexpr int cax(int d) { return d == 0 ? 1 : (d == 1 ? 3 : 9); }

template <bool FORCE, bool FULL, class R>
__device__ __forceinline__ void collide_cumulant(R (&f)[27], const Coll<R> &k, R &rho_out, R &ux_out, R &uy_out,
                                                 R &uz_out)
{
    using L = Lattice<27>;
    R g[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) g[cum_slot(i)] = FULL ? f[i] - R(L::w(i)) : f[i];
    const R r0 = FULL ? R(1) : k.rho0;
    // raw moments along z, y, x
    auto raw = [](R &m, R &z, R &p, int) {
        const R s = p + m, d = p - m;
        const R m0 = s + z;
        m = m0;
        z = d;
        p = s;
    };
    cum_lines<9>(g, raw);
    cum_lines<3>(g, raw);
    cum_lines<1>(g, raw);
    const R drho = g[0];
    const R rho = r0 + drho;
    const R inv = recip(rho);
    R ux, uy, uz;
    if (FORCE) {
        ux = (g[cix(1, 0, 0)] + R(0.5) * k.F[0]) * inv;
        uy = (g[cix(0, 1, 0)] + R(0.5) * k.F[1]) * inv;
        uz = (g[cix(0, 0, 1)] + R(0.5) * k.F[2]) * inv;
    } else {
        ux = g[cix(1, 0, 0)] * inv;
        uy = g[cix(0, 1, 0)] * inv;
        uz = g[cix(0, 0, 1)] * inv;
    }
    rho_out = rho;
    ux_out = ux;
    uy_out = uy;
    uz_out = uz;
    const R third = R(1.0 / 3.0);
    auto c222 = [&](const R (&m)[27], const R (&c4)[27]) {
        const R a = m[cix(2, 0, 0)], b = m[cix(0, 2, 0)], c = m[cix(0, 0, 2)];
        const R xy = m[cix(1, 1, 0)], xz = m[cix(1, 0, 1)], yz = m[cix(0, 1, 1)];
        const R c220 = c4[cix(2, 2, 0)], c202 = c4[cix(2, 0, 2)], c022 = c4[cix(0, 2, 2)];
        const R inv2 = inv * inv;
        R t1 = third * (c022 + c202 + c220) + R(1.0 / 9.0) * (a + b + c);
        R t2 = a * c022 + b * c202 + c * c220 +
               R(4) * (xy * c4[cix(1, 1, 2)] + xz * c4[cix(1, 2, 1)] + yz * c4[cix(2, 1, 1)]) +
               R(2) * (m[cix(2, 1, 0)] * m[cix(0, 1, 2)] + m[cix(2, 0, 1)] * m[cix(0, 2, 1)] + m[cix(1, 2, 0)] * m[cix(1, 0, 2)]) +
               R(4) * m[cix(1, 1, 1)] * m[cix(1, 1, 1)] + third * (a * b + b * c + c * a) +
               R(2.0 / 3.0) * (yz * yz + xz * xz + xy * xy);
        R t3 = a * b * c + R(2) * (a * yz * yz + b * xz * xz + c * xy * xy) + R(8) * xy * xz * yz;
        return t1 + t2 * inv + t3 * inv2;
    };
    // shear and bulk relaxation of the second-order excess (a, b, c, xy, xz, yz)
    auto relax2 = [&](R &a, R &b, R &c, R &xy, R &xz, R &yz) {
        R dxy = a - b, dxz = a - c, tr = a + b + c;
        dxy = fma(-k.cum[0], dxy, dxy);
        dxz = fma(-k.cum[0], dxz, dxz);
        tr = fma(-k.cum[1], tr, tr);
        a = third * (dxy + dxz + tr);
        b = a - dxy;
        c = a - dxz;
        xy = fma(-k.cum[0], xy, xy);
        xz = fma(-k.cum[0], xz, xz);
        yz = fma(-k.cum[0], yz, yz);
    };
    if (k.cum_unit) {
        // every rate beyond the bulk is 1: the cumulants of order 3..6 are reset to zero, so
        // only the second-order excess is needed, from the raw moments:
        //   k^_aa = sum v c_a^2 - drho/3 - rho u_a^2 (+ u_a F_a),
        //   k^_ab = sum v c_a c_b - rho u_a u_b (+ (u_a F_b + u_b F_a)/2)
        R a = fma(-third, drho, g[cix(2, 0, 0)]) - rho * ux * ux;
        R b = fma(-third, drho, g[cix(0, 2, 0)]) - rho * uy * uy;
        R c = fma(-third, drho, g[cix(0, 0, 2)]) - rho * uz * uz;
        R xy = g[cix(1, 1, 0)] - rho * ux * uy, xz = g[cix(1, 0, 1)] - rho * ux * uz, yz = g[cix(0, 1, 1)] - rho * uy * uz;
        if (FORCE) {
            a = fma(ux, k.F[0], a);
            b = fma(uy, k.F[1], b);
            c = fma(uz, k.F[2], c);
            xy += R(0.5) * (ux * k.F[1] + uy * k.F[0]);
            xz += R(0.5) * (ux * k.F[2] + uz * k.F[0]);
            yz += R(0.5) * (uy * k.F[2] + uz * k.F[1]);
        }
        relax2(a, b, c, xy, xz, yz);
        // post-collision excess central moments (orders 3 and 5 vanish with their cumulants)
#pragma unroll
        for (int kk = 0; kk < 27; ++kk) g[kk] = R(0);
        g[cix(2, 0, 0)] = a;
        g[cix(0, 2, 0)] = b;
        g[cix(0, 0, 2)] = c;
        g[cix(1, 1, 0)] = xy;
        g[cix(1, 0, 1)] = xz;
        g[cix(0, 1, 1)] = yz;
        g[cix(2, 2, 2)] = c222(g, g);  // every third- and fourth-order entry still zero here
        g[cix(2, 2, 0)] = third * (a + b) + (a * b + R(2) * xy * xy) * inv;
        g[cix(2, 0, 2)] = third * (a + c) + (a * c + R(2) * xz * xz) * inv;
        g[cix(0, 2, 2)] = third * (b + c) + (b * c + R(2) * yz * yz) * inv;
        g[cix(2, 1, 1)] = third * yz + (a * yz + R(2) * xy * xz) * inv;
        g[cix(1, 2, 1)] = third * xz + (b * xz + R(2) * xy * yz) * inv;
        g[cix(1, 1, 2)] = third * xy + (c * xy + R(2) * xz * yz) * inv;
    } else {
        // central shifts along z, y, x, each adding the equilibrium part r0 W W D(u) it changes
        cum_shift<2, false>(g, uz, r0);
        cum_shift<1, false>(g, uy, r0);
        cum_shift<0, false>(g, ux, r0);
        // excess central moments: remove rho W W W (r0 of it is already out)
#pragma unroll
        for (int kk = 1; kk < 27; ++kk) {
            const double ww = cum_w(kk % 3) * cum_w((kk / 3) % 3) * cum_w(kk / 9);
            if (ww != 0.0) g[kk] = fma(-R(ww), drho, g[kk]);
        }
        // cumulants of order 4..6 (orders 2 and 3: the excess central moments themselves)
        R C[27];
#pragma unroll
        for (int kk = 0; kk < 27; ++kk) C[kk] = g[kk];
        // 211-type: doubled axis d, singles p < q
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int p = d == 0 ? 1 : 0, q = d == 2 ? 1 : 2;
            const int id = 2 * cax(d) + cax(p) + cax(q), pq = cax(p) + cax(q);
            C[id] = g[id] - third * g[pq] - (g[cdd(d)] * g[pq] + R(2) * g[cax(d) + cax(p)] * g[cax(d) + cax(q)]) * inv;
        }
        // 220-type: doubled axes p < q
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int p = s == 0 ? 1 : 0, q = s == 2 ? 1 : 2;
            const int id = 2 * cax(p) + 2 * cax(q);
            C[id] = g[id] - third * (g[cdd(p)] + g[cdd(q)]) - (g[cdd(p)] * g[cdd(q)] + R(2) * g[cax(p) + cax(q)] * g[cax(p) + cax(q)]) * inv;
        }
        // 122-type: single axis s, doubled p < q
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int p = s == 0 ? 1 : 0, q = s == 2 ? 1 : 2;
            const int id = cax(s) + 2 * cax(p) + 2 * cax(q);
            const int s2q = cax(s) + 2 * cax(q), s2p = cax(s) + 2 * cax(p);
            C[id] = g[id] - third * (g[s2q] + g[s2p]) -
                    (g[cdd(p)] * g[s2q] + g[cdd(q)] * g[s2p] + R(2) * g[cax(s) + cax(p)] * g[cax(p) + 2 * cax(q)] +
                     R(2) * g[cax(s) + cax(q)] * g[2 * cax(p) + cax(q)] + R(4) * g[cax(p) + cax(q)] * g[cix(1, 1, 1)]) *
                        inv;
        }
        C[cix(2, 2, 2)] = g[cix(2, 2, 2)] - c222(g, C);
        // relaxation
        const R *w = k.cum;  // shear, bulk, 3 sum, 3 diff, 111, 4 diff, 4 sum, 211, 5th, 6th
        relax2(C[cix(2, 0, 0)], C[cix(0, 2, 0)], C[cix(0, 0, 2)], C[cix(1, 1, 0)], C[cix(1, 0, 1)], C[cix(0, 1, 1)]);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int p = s == 0 ? 1 : 0, q = s == 2 ? 1 : 2;
            const int A = cax(s) + 2 * cax(p), B = cax(s) + 2 * cax(q);
            R sm = C[A] + C[B], df = C[A] - C[B];
            sm = fma(-w[2], sm, sm);
            df = fma(-w[3], df, df);
            C[A] = R(0.5) * (sm + df);
            C[B] = R(0.5) * (sm - df);
        }
        C[cix(1, 1, 1)] = fma(-w[4], C[cix(1, 1, 1)], C[cix(1, 1, 1)]);
        {
            const R a = C[cix(2, 2, 0)], b = C[cix(2, 0, 2)], c = C[cix(0, 2, 2)];
            R d1 = a - R(2) * b + c, d2 = a + b - R(2) * c, t = a + b + c;
            d1 = fma(-w[5], d1, d1);
            d2 = fma(-w[5], d2, d2);
            t = fma(-w[6], t, t);
            C[cix(2, 2, 0)] = third * (d1 + d2 + t);
            C[cix(2, 0, 2)] = third * (t - d1);
            C[cix(0, 2, 2)] = third * (t - d2);
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int id = cax(d) + 13;  // 2 cax(d) + the two other axes once (1 + 3 + 9 - cax(d))
            C[id] = fma(-w[7], C[id], C[id]);
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int id = 26 - cax(s);  // cax(s) + the two other axes twice, 2 (13 - cax(s))
            C[id] = fma(-w[8], C[id], C[id]);
        }
        C[cix(2, 2, 2)] = fma(-w[9], C[cix(2, 2, 2)], C[cix(2, 2, 2)]);
        // back to excess central moments, in order of increasing order
#pragma unroll
        for (int kk = 0; kk < 27; ++kk) g[kk] = C[kk];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int p = d == 0 ? 1 : 0, q = d == 2 ? 1 : 2;
            const int id = 2 * cax(d) + cax(p) + cax(q), pq = cax(p) + cax(q);
            g[id] = C[id] + third * C[pq] + (C[cdd(d)] * C[pq] + R(2) * C[cax(d) + cax(p)] * C[cax(d) + cax(q)]) * inv;
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int p = s == 0 ? 1 : 0, q = s == 2 ? 1 : 2;
            const int id = 2 * cax(p) + 2 * cax(q);
            g[id] = C[id] + third * (C[cdd(p)] + C[cdd(q)]) + (C[cdd(p)] * C[cdd(q)] + R(2) * C[cax(p) + cax(q)] * C[cax(p) + cax(q)]) * inv;
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int p = s == 0 ? 1 : 0, q = s == 2 ? 1 : 2;
            const int id = cax(s) + 2 * cax(p) + 2 * cax(q);
            const int s2q = cax(s) + 2 * cax(q), s2p = cax(s) + 2 * cax(p);
            g[id] = C[id] + third * (C[s2q] + C[s2p]) +
                    (C[cdd(p)] * C[s2q] + C[cdd(q)] * C[s2p] + R(2) * C[cax(s) + cax(p)] * C[cax(p) + 2 * cax(q)] +
                     R(2) * C[cax(s) + cax(q)] * C[2 * cax(p) + cax(q)] + R(4) * C[cax(p) + cax(q)] * C[cix(1, 1, 1)]) *
                        inv;
        }
        g[cix(2, 2, 2)] = C[cix(2, 2, 2)] + c222(C, C);
    }
    // central moments less r0 W W W: add rho - r0 of W W W back; first order +F/2
#pragma unroll
    for (int kk = 1; kk < 27; ++kk) {
        const double ww = cum_w(kk % 3) * cum_w((kk / 3) % 3) * cum_w(kk / 9);
        if (ww != 0.0) g[kk] = fma(R(ww), drho, g[kk]);
    }
    g[0] = drho;
    g[cix(1, 0, 0)] = FORCE ? R(0.5) * k.F[0] : R(0);
    g[cix(0, 1, 0)] = FORCE ? R(0.5) * k.F[1] : R(0);
    g[cix(0, 0, 1)] = FORCE ? R(0.5) * k.F[2] : R(0);
    // inverse central shifts x, y, z (the forward order reversed)
    cum_shift<0, true>(g, ux, r0);
    cum_shift<1, true>(g, uy, r0);
    cum_shift<2, true>(g, uz, r0);
    // raw moments back to populations
    auto raw_back = [](R &m0, R &m1, R &m2, int) {
        const R p0 = m0 - m2;
        const R pp = R(0.5) * (m2 + m1), pm = R(0.5) * (m2 - m1);
        m0 = pm;
        m1 = p0;
        m2 = pp;
    };
    cum_lines<1>(g, raw_back);
    cum_lines<3>(g, raw_back);
    cum_lines<9>(g, raw_back);
#pragma unroll
    for (int i = 0; i < 27; ++i) f[i] = FULL ? g[cum_slot(i)] + R(L::w(i)) : g[cum_slot(i)];
}

}  // namespace lbm
