// D3Q15 / D3Q19 velocity sets of libhemelb_gb300 as constexpr arithmetic, so
// that unrolled device loops fold every c_i component and weight into an
// immediate (no tables in memory).
//
// Direction order: 0 = rest; 1..6 = +x -x +y -y +z -z; then pairs of
// opposite vectors, odd index = the pair's base vector, even = its negative:
//   D3Q15 bases (1,1,1) (1,1,-1) (1,-1,1) (-1,1,1)
//   D3Q19 bases (1,1,0) (1,-1,0) (1,0,1) (1,0,-1) (0,1,1) (0,1,-1)
// Weights (textbook, fixed by lattice isotropy): D3Q15 2/9, 1/9, 1/72;
// D3Q19 1/3, 1/18, 1/36 for |c|^2 = 0, 1, and 3 resp. 2.
#pragma once

#if defined(__CUDACC__)
#define HGB_HD __host__ __device__ __forceinline__
#else
#define HGB_HD inline
#endif

namespace hemelb_gb300 {

template <int Q>
HGB_HD constexpr int cdir(int i, int a) {
    if (i == 0) return 0;
    if (i <= 6) return (a == ((i - 1) >> 1)) ? ((i & 1) ? 1 : -1) : 0;
    const int p = (i - 7) >> 1;
    const int sg = (i & 1) ? 1 : -1;
    if (Q == 15) {
        const int neg_axis = p == 1 ? 2 : (p == 2 ? 1 : (p == 3 ? 0 : -1));
        return sg * (a == neg_axis ? -1 : 1);
    }
    const int zero_axis = p < 2 ? 2 : (p < 4 ? 1 : 0);
    if (a == zero_axis) return 0;
    const int first = zero_axis == 0 ? 1 : 0;
    return sg * ((a == first) ? 1 : ((p & 1) ? -1 : 1));
}

HGB_HD constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

template <int Q>
HGB_HD constexpr int clen2(int i) {
    return cdir<Q>(i, 0) * cdir<Q>(i, 0) + cdir<Q>(i, 1) * cdir<Q>(i, 1) +
           cdir<Q>(i, 2) * cdir<Q>(i, 2);
}

template <int Q>
HGB_HD constexpr double wdir(int i) {
    return Q == 15 ? (clen2<Q>(i) == 0 ? 2.0 / 9.0 : (clen2<Q>(i) == 1 ? 1.0 / 9.0 : 1.0 / 72.0))
                   : (clen2<Q>(i) == 0 ? 1.0 / 3.0 : (clen2<Q>(i) == 1 ? 1.0 / 18.0 : 1.0 / 36.0));
}

// runtime-q versions for host code
HGB_HD int cdir_q(int q, int i, int a) { return q == 15 ? cdir<15>(i, a) : cdir<19>(i, a); }
HGB_HD double wdir_q(int q, int i) { return q == 15 ? wdir<15>(i) : wdir<19>(i); }

}  // namespace hemelb_gb300
