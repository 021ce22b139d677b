// lattice.cuh -- D3Q19 / D3Q27 velocity sets for the CUDA path (host and device).
//
// The paper names both stencils (Sec. 5.1.1) without printing a table.  These are
// the standard tables (c_s^2 = 1/3) in the library's canonical order: rest; +x -x +y -y +z -z;
// the 12 |c|^2 = 2 vectors in lexicographic (cx, cy, cz) order; for D3Q27 the 8 corners in
// lexicographic order.  Opposite pairs: (1,2) (3,4) (5,6), edges i <-> 25 - i, corners
// i <-> 45 - i.  Accessors are constexpr functions so that unrolled device loops fold them
// into immediates.
#pragma once

#include <cstdint>

namespace lbm {

template <int Q>
struct Lattice;

template <>
struct Lattice<19> {
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, -1, -1, -1, -1, 0, 0, 0, 0, 1, 1, 1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, -1, 0, 0, 1, -1, -1, 1, 1, -1, 0, 0, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, -1, 1, 0, -1, 1, -1, 1, 0, -1, 1, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : 25 - i);
    }
    // weights by |c|^2: 0 -> 1/3, 1 -> 1/18, 2 -> 1/36
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 1.0 / 3 : (i <= 6 ? 1.0 / 18 : 1.0 / 36); }
};

template <>
struct Lattice<27> {
    static constexpr int Q = 27;
    __host__ __device__ static constexpr int cx(int i)
    {
        constexpr int t[27] = {0, 1, -1, 0, 0, 0, 0, -1, -1, -1, -1, 0, 0, 0,
                               0, 1, 1,  1, 1, -1, -1, -1, -1, 1, 1, 1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        constexpr int t[27] = {0, 0, 0, 1, -1, 0, 0, -1, 0, 0, 1, -1, -1, 1,
                               1, -1, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        constexpr int t[27] = {0, 0, 0, 0, 0, 1, -1, 0, -1, 1, 0, -1, 1, -1,
                               1, 0, -1, 1, 0, -1, 1, -1, 1, -1, 1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int opp(int i)
    {
        return i == 0 ? 0 : (i <= 6 ? ((i & 1) ? i + 1 : i - 1) : (i <= 18 ? 25 - i : 45 - i));
    }
    // weights by |c|^2: 0 -> 8/27, 1 -> 2/27, 2 -> 1/54, 3 -> 1/216
    __host__ __device__ static constexpr double w(int i)
    {
        return i == 0 ? 8.0 / 27 : (i <= 6 ? 2.0 / 27 : (i <= 18 ? 1.0 / 54 : 1.0 / 216));
    }
};

// Runtime tables for host code (list builder), which handles both stencils.
struct LatticeView {
    int q;
    int cx[27], cy[27], cz[27], opp[27];
    double w[27];
};

template <int Q>
inline LatticeView make_view()
{
    LatticeView v{};
    v.q = Q;
    for (int i = 0; i < Q; ++i) {
        v.cx[i] = Lattice<Q>::cx(i);
        v.cy[i] = Lattice<Q>::cy(i);
        v.cz[i] = Lattice<Q>::cz(i);
        v.opp[i] = Lattice<Q>::opp(i);
        v.w[i] = Lattice<Q>::w(i);
    }
    return v;
}

inline LatticeView lattice_view(int q) { return q == 27 ? make_view<27>() : make_view<19>(); }

}  // namespace lbm
