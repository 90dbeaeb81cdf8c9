// CUDA kernels of libhemelb_gb300 (sm_103a) around the step (the step
// kernels themselves are in lbm_step.cu): the macroscopic fields and wall
// shear stress, the float64 mass reduction, the gather/scatter that convert
// the stored state to and from caller-order float64 populations, and the
// exact layout conversion between pull and AA storage.
//
// The method (arXiv 1906.11925, Section 2): collision then propagation of a
// single-particle distribution on a sparse lattice of fluid sites, D3Q19
// (Fig. 1); simple bounce-back walls (Section 4).  Collision is LBGK with the
// compressible second-order equilibrium; iolets impose a density through the
// equilibrium populations entering from the iolet (see lbm.h).
//
// Storage: the buffer read at step t holds, for every site x and direction i,
// the slot P_i(x) that the pull of step t reads; this is the post-collision
// population f*_i(x, t-1) for fluid and wall links, and for an iolet link the
// equilibrium population already evaluated at the iolet density.  Reading
// the slots through the table (lbm_internal.h) is a permutation, so the
// gather reproduces f(t) exactly.  Values are deviations d = f - w_i rho0,
// in float or in IEEE half scaled by 2^S.
//
// The step is a bandwidth-bound sparse stencil (about one flop per byte): no
// tensor cores.  One site per thread; the q - 1 table entries are streamed
// (evict-first) and coalesced; the q population reads are gathers through the
// read-only path, made local by the Morton order; the q stores are coalesced
// and streamed.
#include <cuda_fp16.h>

#include <algorithm>

#include "lattice.h"
#include "lbm_internal.h"

namespace hemelb_gb300 {
namespace {

constexpr int kBlock = 256;
constexpr int kMassBlocks = 2 * 152;  // fixed grid: deterministic reduction order
template <int HALF>
struct Store;

template <>
struct Store<0> {
    using T = float;
    static __device__ __forceinline__ float load(const float *p, float) { return __ldg(p); }
    static __device__ __forceinline__ float load_plain(const float *p, float) { return *p; }
    static __device__ __forceinline__ void store(float *p, float v, float) { __stcs(p, v); }
    static __device__ __forceinline__ void store_plain(float *p, float v, float) { *p = v; }
};

template <>
struct Store<1> {
    using T = __half;
    static __device__ __forceinline__ float load(const __half *p, float inv) {
        return __half2float(__ldg(p)) * inv;
    }
    static __device__ __forceinline__ float load_plain(const __half *p, float inv) {
        return __half2float(*p) * inv;
    }
    static __device__ __forceinline__ void store(__half *p, float v, float sc) {
        __stcs(reinterpret_cast<short *>(p), __half_as_short(__float2half_rn(v * sc)));
    }
    static __device__ __forceinline__ void store_plain(__half *p, float v, float sc) {
        *p = __float2half_rn(v * sc);
    }
};

// int16 fixed point: value = round(deviation 2^S), |value| <= 32766; the
// saturation codes +-32767 read as NaN (an out-of-range state shows as
// non-finite, as an fp16 overflow does), -32768 is the guard code.
__device__ __forceinline__ float i16_value(int v, float inv) {
    return (v >= 32767 || v <= -32767) ? __int_as_float(0x7fc00000) : (__int_as_float(0x4B400000 + v) - 12582912.0f) * inv;
}
__device__ __forceinline__ short i16_code(float v) {
    const float c = fminf(fmaxf(v, -32767.0f), 32767.0f);
    return (short)(__float_as_int(c + 12582912.0f) - 0x4B400000);
}
template <>
struct Store<2> {
    using T = short;
    static __device__ __forceinline__ float load(const short *p, float inv) { return i16_value(__ldg(p), inv); }
    static __device__ __forceinline__ float load_plain(const short *p, float inv) { return i16_value(*p, inv); }
    static __device__ __forceinline__ void store(short *p, float v, float sc) { __stcs(p, i16_code(v * sc)); }
    static __device__ __forceinline__ void store_plain(short *p, float v, float sc) { *p = i16_code(v * sc); }
};

// Slot holding population i of site x (table entry s) in each layout:
//   pull        P[i][s] (the site x - c_i), or P[opp(i)][x] for a wall/iolet link;
//   natural     A[i][x] (AA pattern after an odd step);
//   AA swapped  A[opp(i)][s], or A[i][x] for a wall/iolet link (after an even step).
__device__ __forceinline__ int64_t src_slot(int layout, int i, int s, int x, int64_t np) {
    if (layout == LAYOUT_NATURAL) return (int64_t)i * np + x;
    const int a = layout == LAYOUT_PULL ? i : opp(i);
    const int b = layout == LAYOUT_PULL ? opp(i) : i;
    return s >= 0 ? (int64_t)a * np + s : (int64_t)b * np + x;
}

// Gather the q deviations of site x (pre-collision populations f(t) - w rho0).
// Returns the smallest table entry seen and, through wall_n, the sum of c_i
// over wall entries (half-way or interpolated).
template <int Q, int HALF, bool STREAM_TAB, bool BFL = false>
__device__ __forceinline__ int gather(const DevLattice &L, const typename Store<HALF>::T *__restrict__ f,
                                      int layout, int x, float (&d)[Q], int (&wn)[3]) {
    using S = Store<HALF>;
    const int64_t np = L.npad;
    int minc = 0;
    wn[0] = wn[1] = wn[2] = 0;
    int s[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int32_t *tp = L.tab + (int64_t)(i - 1) * np + x;
        s[i] = STREAM_TAB ? __ldcs(tp) : __ldg(tp);
    }
    d[0] = S::load(f + x, L.inv_scale);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        d[i] = S::load(f + src_slot(layout, i, s[i], x, np), L.inv_scale);
        minc = min(minc, s[i]);
        // (without interpolated walls the is_bfl test never holds; for float
        // storage the compiler schedules this form faster: 0.43 ms instead of
        // 0.61 ms for the fields of the 10.8M-site tree, 0.52 instead of 0.80
        // for its wall-shear-stress volume)
        if (s[i] == -1 || ((BFL || !HALF) && is_bfl(s[i]))) {
            wn[0] += cdir<Q>(i, 0);
            wn[1] += cdir<Q>(i, 1);
            wn[2] += cdir<Q>(i, 2);
        }
    }
    if (BFL && x >= L.n_bulk) {
        // interpolated walls (every layout): q < 1/2 with a fluid
        // upstream site adds (1 - 2q) times the population pulled from it
#pragma unroll
        for (int p = 1; p < Q; ++p)
            if (is_bfl(s[p])) {
                const float qv = bfl_q(s[p]);
                if (qv < 0.5f && s[opp(p)] >= 0) d[p] = fmaf(1.0f - 2.0f * qv, d[opp(p)], d[p]);
            }
    }
    return minc;
}

struct Moments {
    float drho, rho, ux, uy, uz, usq15;
};

template <int Q>
__device__ __forceinline__ Moments moments(const float (&d)[Q], float rho0) {
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        drho += d[i];
        if (cdir<Q>(i, 0)) jx += cdir<Q>(i, 0) * d[i];
        if (cdir<Q>(i, 1)) jy += cdir<Q>(i, 1) * d[i];
        if (cdir<Q>(i, 2)) jz += cdir<Q>(i, 2) * d[i];
    }
    Moments m;
    m.drho = drho;
    m.rho = rho0 + drho;
    const float ir = 1.0f / m.rho;
    m.ux = jx * ir;
    m.uy = jy * ir;
    m.uz = jz * ir;
    m.usq15 = 1.5f * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    return m;
}

// deviation of the equilibrium: feq_i - w_i rho0 = w_i (drho + rho A_i)
template <int Q>
__device__ __forceinline__ float deq(int i, float drho, float rho, const Moments &m) {
    const float cu = cdir<Q>(i, 0) * m.ux + cdir<Q>(i, 1) * m.uy + cdir<Q>(i, 2) * m.uz;
    return (float)wdir<Q>(i) * (drho + rho * (3.0f * cu + 4.5f * cu * cu - m.usq15));
}

// Wall shear stress of a site from its deviations, moments and the sum of
// c_i over its wall links (0 when the site has no wall links or they sum to 0).
template <int Q>
__device__ __forceinline__ float wall_shear(const float (&d)[Q], const Moments &m, const int (&wn)[3],
                                            float tau) {
    // sum of c over wall links = -(sum of c_i over entries -1); n = -normalize()
    const float nn2 = (float)(wn[0] * wn[0] + wn[1] * wn[1] + wn[2] * wn[2]);
    if (nn2 == 0.f) return 0.f;
    const float inn = 1.0f / sqrtf(nn2);
    const float n0 = wn[0] * inn, n1 = wn[1] * inn, n2 = wn[2] * inn;
    float pxx = 0.f, pyy = 0.f, pzz = 0.f, pxy = 0.f, pxz = 0.f, pyz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const float ne = d[i] - deq<Q>(i, m.drho, m.rho, m);
        const int cx = cdir<Q>(i, 0), cy = cdir<Q>(i, 1), cz = cdir<Q>(i, 2);
        if (cx) pxx += ne;
        if (cy) pyy += ne;
        if (cz) pzz += ne;
        if (cx * cy) pxy += (cx * cy) * ne;
        if (cx * cz) pxz += (cx * cz) * ne;
        if (cy * cz) pyz += (cy * cz) * ne;
    }
    const float coef = -(1.0f - 0.5f / tau);
    const float t0 = coef * (pxx * n0 + pxy * n1 + pxz * n2);
    const float t1 = coef * (pxy * n0 + pyy * n1 + pyz * n2);
    const float t2 = coef * (pxz * n0 + pyz * n1 + pzz * n2);
    const float tn = t0 * n0 + t1 * n1 + t2 * n2;
    const float s0 = t0 - tn * n0, s1 = t1 - tn * n1, s2 = t2 - tn * n2;
    return sqrtf(s0 * s0 + s1 * s1 + s2 * s2);
}

#ifndef HGB_MACROS_MINB
#define HGB_MACROS_MINB 3
#endif
template <int Q, int HALF, bool BFL>
__global__ void __launch_bounds__(kBlock, HGB_MACROS_MINB)
k_macros(const DevLattice L, const typename Store<HALF>::T *__restrict__ f, int layout,
         float *__restrict__ rho, float *__restrict__ u, float *__restrict__ wss) {
    const int x = blockIdx.x * kBlock + threadIdx.x;
    if (x >= L.n) return;
    float d[Q];
    int wn[3];
    gather<Q, HALF, false, BFL>(L, f, layout, x, d, wn);
    const Moments m = moments<Q>(d, L.rho0);
    const int xc = L.perm[x];
    if (rho) rho[xc] = m.rho;
    if (u) {
        u[3 * (int64_t)xc + 0] = m.ux;
        u[3 * (int64_t)xc + 1] = m.uy;
        u[3 * (int64_t)xc + 2] = m.uz;
    }
    if (wss) wss[xc] = wall_shear<Q>(d, m, wn, L.tau);
}

// Quantity of site x written into the render volume through a surface at
// voxel coordinates (packed 21 bits per axis, relative to the lattice's box)
// plus shift; sites outside the volume are skipped.  With mark set, every
// 8^3 brick whose samples can depend on the voxel (voxel index within
// [8b - 2, 8b + 9] on each axis) is flagged non-empty.
#ifndef HGB_FILL_MINB
#define HGB_FILL_MINB 3
#endif
template <int Q, int HALF, int QTY, bool BFL>
__global__ void __launch_bounds__(kBlock, QTY == 2 ? 1 : HGB_FILL_MINB)
k_volume_fill(const DevLattice L, const typename Store<HALF>::T *__restrict__ f, int layout,
              const uint64_t *__restrict__ vox, VolumeTarget V) {
    const int x = blockIdx.x * kBlock + threadIdx.x;
    if (x >= L.n) return;
    const uint64_t pk = vox[x];
    const int vx = (int)(pk & 0x1fffff) + V.shift[0];
    const int vy = (int)((pk >> 21) & 0x1fffff) + V.shift[1];
    const int vz = (int)((pk >> 42) & 0x1fffff) + V.shift[2];
    if (vx < 0 || vy < 0 || vz < 0 || vx >= V.dims[0] || vy >= V.dims[1] || vz >= V.dims[2]) return;
    float d[Q];
    int wn[3];
    gather<Q, HALF, false, BFL>(L, f, layout, x, d, wn);
    const Moments m = moments<Q>(d, L.rho0);
    float v;
    if (QTY == 0)
        v = m.rho;
    else if (QTY == 1)
        v = sqrtf(m.ux * m.ux + m.uy * m.uy + m.uz * m.uz);
    else
        v = wall_shear<Q>(d, m, wn, L.tau);
    surf3Dwrite(v, V.surf, vx * (int)sizeof(float), vy, vz, cudaBoundaryModeZero);
    if (!V.mark) return;
    const int p[3] = {vx, vy, vz};
    int b0[3], b1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b0[a] = max(0, (p[a] - 9 + 7) >> 3);  // ceil((p - 9) / 8), p - 9 + 7 >= -9: >> floors
        b1[a] = min(V.bdims[a] - 1, (p[a] + 2) >> 3);
    }
    for (int bz = b0[2]; bz <= b1[2]; ++bz)
        for (int by = b0[1]; by <= b1[1]; ++by)
            for (int bx = b0[0]; bx <= b1[0]; ++bx)
                V.occ[((int64_t)bz * V.bdims[1] + by) * V.bdims[0] + bx] = 1;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block sum in a fixed order; result valid in thread 0
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double part[kBlock / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = threadIdx.x < kBlock / 32 ? part[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

// mass = n rho0 + sum over all stored slots of the deviation: the gather is a
// permutation of the slots, so the slots hold exactly the populations f(t).
template <int Q, int HALF, bool BFL>
__global__ void __launch_bounds__(kBlock)
k_mass_partial(const DevLattice L, const typename Store<HALF>::T *__restrict__ f, int layout,
               double *__restrict__ partials) {
    using S = Store<HALF>;
    double acc = 0.0;
    for (int x = blockIdx.x * kBlock + threadIdx.x; x < L.n; x += gridDim.x * kBlock) {
        // the q slots of a site are summed in float (deviations, ~1e-3 of
        // the density), the sites in float64: float64 per slot costs q double
        // additions per site, several times the time of reading the slots
        float s = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) s += S::load(f + (int64_t)i * L.npad + x, L.inv_scale);
        if (BFL && x >= L.n_bulk) {
            // interpolated walls: the slot of a q < 1/2 link holds only part of
            // the population; the rest is (1 - 2q) times the population opp(p)
            // that the site gathers from its upstream neighbour (in the slot
            // the layout keeps it in)
#pragma unroll
            for (int p = 1; p < Q; ++p) {
                const int e = L.tab[(int64_t)(p - 1) * L.npad + x];
                if (!is_bfl(e)) continue;
                const float qv = bfl_q(e);
                const int u = L.tab[(int64_t)(opp(p) - 1) * L.npad + x];
                if (qv < 0.5f && u >= 0)
                    s += (1.0f - 2.0f * qv) * S::load(f + src_slot(layout, opp(p), u, x, L.npad), L.inv_scale);
            }
        }
        acc += (double)s;
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kBlock)
k_mass_final(const double *__restrict__ partials, int nparts, double base, double *__restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < nparts; i += kBlock) acc += partials[i];
    acc = block_sum(acc);
    if (threadIdx.x == 0) out[0] = base + acc;
}

// Weighted sum over the sites of q(x) (KIND 0: wall shear stress, 1:
// density), per-block float64 partial sums in a fixed grid (deterministic):
// weight is float64 in caller order (null: all ones).  The density is formed
// as rho0 + drho in float64 so that the deviation keeps its precision.
template <int Q, int HALF, int KIND, bool BFL>
__global__ void __launch_bounds__(kBlock)
k_wsum_partial(const DevLattice L, const typename Store<HALF>::T *__restrict__ f, int layout,
               const double *__restrict__ weight, double *__restrict__ partials) {
    double acc = 0.0;
    for (int x = blockIdx.x * kBlock + threadIdx.x; x < L.n; x += gridDim.x * kBlock) {
        const double w = weight ? weight[L.perm[x]] : 1.0;
        if (w == 0.0) continue;
        float d[Q];
        int wn[3];
        gather<Q, HALF, false, BFL>(L, f, layout, x, d, wn);
        const Moments m = moments<Q>(d, L.rho0);
        if (KIND == 1)
            acc += w * ((double)L.rho0 + (double)m.drho);
        else
            acc += w * (double)wall_shear<Q>(d, m, wn, L.tau);
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

template <int Q, int HALF, bool BFL>
__global__ void __launch_bounds__(kBlock)
k_gather_f64(const DevLattice L, const typename Store<HALF>::T *__restrict__ f, int layout,
             double *__restrict__ out) {
    const int x = blockIdx.x * kBlock + threadIdx.x;
    if (x >= L.n) return;
    float d[Q];
    int wn[3];
    gather<Q, HALF, false, BFL>(L, f, layout, x, d, wn);
    const int64_t xc = L.perm[x];
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(int64_t)i * L.n + xc] = wdir<Q>(i) * (double)L.rho0 + (double)d[i];
}

template <int Q, int HALF>
__global__ void __launch_bounds__(kBlock)
k_scatter_f64(const DevLattice L, const double *__restrict__ in, int layout,
              typename Store<HALF>::T *__restrict__ f) {
    using S = Store<HALF>;
    const int x = blockIdx.x * kBlock + threadIdx.x;
    if (x >= L.n) return;
    const int64_t xc = L.perm[x];
    const int64_t np = L.npad;
    S::store_plain(f + x, (float)(in[xc] - wdir<Q>(0) * (double)L.rho0), L.scale);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int s = L.tab[(int64_t)(i - 1) * np + x];
        double v = in[(int64_t)i * L.n + xc] - wdir<Q>(i) * (double)L.rho0;
        if (is_bfl(s)) {
            // the slot keeps f_i - (1 - 2q) f_opp(i) when the gather adds the rest
            const double qv = bfl_q(s);
            if (qv < 0.5 && L.tab[(int64_t)(opp(i) - 1) * np + x] >= 0)
                v -= (1.0 - 2.0 * qv) * (in[(int64_t)opp(i) * L.n + xc] - wdir<Q>(i) * (double)L.rho0);
        }
        S::store_plain(f + src_slot(layout, i, s, x, np), (float)v, L.scale);
    }
}

// Exact copy of the stored state from one layout to another (a permutation of
// the stored elements; no arithmetic).
template <typename T, int Q>
__global__ void __launch_bounds__(kBlock)
k_relayout(const DevLattice L, const T *__restrict__ src, int src_layout, T *__restrict__ dst,
           int dst_layout) {
    const int x = blockIdx.x * kBlock + threadIdx.x;
    if (x >= L.n) return;
    const int64_t np = L.npad;
    dst[x] = src[x];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int s = L.tab[(int64_t)(i - 1) * np + x];
        dst[src_slot(dst_layout, i, s, x, np)] = src[src_slot(src_layout, i, s, x, np)];
    }
}

inline unsigned grid_for(int n) { return (unsigned)((n + kBlock - 1) / kBlock); }

}  // namespace

#define HGB_DISPATCH(L, FN, ...)                                                         \
    ((L).q == 15 ? ((L).storage == 2 ? FN<15, 2>(__VA_ARGS__)                                 \
                                     : (L).storage ? FN<15, 1>(__VA_ARGS__) : FN<15, 0>(__VA_ARGS__)) \
                 : ((L).storage == 2 ? FN<19, 2>(__VA_ARGS__)                                 \
                                     : (L).storage ? FN<19, 1>(__VA_ARGS__) : FN<19, 0>(__VA_ARGS__)))

cudaError_t launch_relayout(const DevLattice &L, const void *src, int src_layout, void *dst,
                            int dst_layout, cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    if (L.storage) {
        if (L.q == 15)
            k_relayout<short, 15><<<grid_for(L.n), kBlock, 0, s>>>(L, (const short *)src, src_layout, (short *)dst, dst_layout);
        else
            k_relayout<short, 19><<<grid_for(L.n), kBlock, 0, s>>>(L, (const short *)src, src_layout, (short *)dst, dst_layout);
    } else {
        if (L.q == 15)
            k_relayout<float, 15><<<grid_for(L.n), kBlock, 0, s>>>(L, (const float *)src, src_layout, (float *)dst, dst_layout);
        else
            k_relayout<float, 19><<<grid_for(L.n), kBlock, 0, s>>>(L, (const float *)src, src_layout, (float *)dst, dst_layout);
    }
    return cudaGetLastError();
}

namespace {
template <int Q, int HALF>
cudaError_t macros_impl(const DevLattice &L, const void *f, int layout, float *rho, float *u, float *wss,
                        cudaStream_t s) {
    using T = typename Store<HALF>::T;
    if (L.bfl)
        k_macros<Q, HALF, true><<<grid_for(L.n), kBlock, 0, s>>>(L, (const T *)f, layout, rho, u, wss);
    else
        k_macros<Q, HALF, false><<<grid_for(L.n), kBlock, 0, s>>>(L, (const T *)f, layout, rho, u, wss);
    return cudaGetLastError();
}
template <int Q, int HALF>
cudaError_t mass_impl(const DevLattice &L, const void *f, int layout, double *partials, cudaStream_t s) {
    using T = typename Store<HALF>::T;
    if (L.bfl)
        k_mass_partial<Q, HALF, true><<<kMassBlocks, kBlock, 0, s>>>(L, (const T *)f, layout, partials);
    else
        k_mass_partial<Q, HALF, false><<<kMassBlocks, kBlock, 0, s>>>(L, (const T *)f, layout, partials);
    return cudaGetLastError();
}
template <int Q, int HALF>
cudaError_t gather_impl(const DevLattice &L, const void *f, int layout, double *out, cudaStream_t s) {
    using T = typename Store<HALF>::T;
    if (L.bfl)
        k_gather_f64<Q, HALF, true><<<grid_for(L.n), kBlock, 0, s>>>(L, (const T *)f, layout, out);
    else
        k_gather_f64<Q, HALF, false><<<grid_for(L.n), kBlock, 0, s>>>(L, (const T *)f, layout, out);
    return cudaGetLastError();
}
template <int Q, int HALF>
cudaError_t scatter_impl(const DevLattice &L, const double *in, int layout, void *f, cudaStream_t s) {
    using T = typename Store<HALF>::T;
    k_scatter_f64<Q, HALF><<<grid_for(L.n), kBlock, 0, s>>>(L, in, layout, (T *)f);
    return cudaGetLastError();
}
template <int Q, int HALF>
cudaError_t volume_fill_impl(const DevLattice &L, const void *f, int layout, const uint64_t *vox,
                             const VolumeTarget &V, cudaStream_t s) {
    using T = typename Store<HALF>::T;
    const unsigned g = grid_for(L.n);
    const T *ft = (const T *)f;
    if (L.bfl) {
        if (V.quantity == 0) k_volume_fill<Q, HALF, 0, true><<<g, kBlock, 0, s>>>(L, ft, layout, vox, V);
        else if (V.quantity == 1) k_volume_fill<Q, HALF, 1, true><<<g, kBlock, 0, s>>>(L, ft, layout, vox, V);
        else k_volume_fill<Q, HALF, 2, true><<<g, kBlock, 0, s>>>(L, ft, layout, vox, V);
    } else {
        if (V.quantity == 0) k_volume_fill<Q, HALF, 0, false><<<g, kBlock, 0, s>>>(L, ft, layout, vox, V);
        else if (V.quantity == 1) k_volume_fill<Q, HALF, 1, false><<<g, kBlock, 0, s>>>(L, ft, layout, vox, V);
        else k_volume_fill<Q, HALF, 2, false><<<g, kBlock, 0, s>>>(L, ft, layout, vox, V);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_volume_fill(const DevLattice &L, const void *f, int layout, const uint64_t *vox,
                               const VolumeTarget &V, cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, volume_fill_impl, L, f, layout, vox, V, s);
}

cudaError_t launch_macros(const DevLattice &L, const void *f, int layout, float *rho, float *u,
                          float *wss, cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, macros_impl, L, f, layout, rho, u, wss, s);
}

namespace {
template <int Q, int HALF>
cudaError_t wsum_impl(const DevLattice &L, const void *f, int layout, int kind, const double *weight,
                      double *partials, cudaStream_t s) {
    using T = typename Store<HALF>::T;
    const T *ft = (const T *)f;
    if (L.bfl) {
        if (kind == 1) k_wsum_partial<Q, HALF, 1, true><<<kMassBlocks, kBlock, 0, s>>>(L, ft, layout, weight, partials);
        else k_wsum_partial<Q, HALF, 0, true><<<kMassBlocks, kBlock, 0, s>>>(L, ft, layout, weight, partials);
    } else {
        if (kind == 1) k_wsum_partial<Q, HALF, 1, false><<<kMassBlocks, kBlock, 0, s>>>(L, ft, layout, weight, partials);
        else k_wsum_partial<Q, HALF, 0, false><<<kMassBlocks, kBlock, 0, s>>>(L, ft, layout, weight, partials);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_weighted_sum(const DevLattice &L, const void *f, int layout, int kind,
                                const double *weight, double *partials, double *out, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    if (L.n > 0) e = HGB_DISPATCH(L, wsum_impl, L, f, layout, kind, weight, partials, s);
    else e = cudaMemsetAsync(partials, 0, (size_t)kMassBlocks * 8, s);
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, kBlock, 0, s>>>(partials, kMassBlocks, 0.0, out);
    return cudaGetLastError();
}

int mass_blocks() { return kMassBlocks; }

cudaError_t launch_mass(const DevLattice &L, const void *f, int layout, double *partials, double *out,
                        cudaStream_t s) {
    cudaError_t e = HGB_DISPATCH(L, mass_impl, L, f, layout, partials, s);
    if (e != cudaSuccess) return e;
    k_mass_final<<<1, kBlock, 0, s>>>(partials, kMassBlocks, (double)L.n * (double)L.rho0, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_f64(const DevLattice &L, const void *f, int layout, double *out,
                              cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, gather_impl, L, f, layout, out, s);
}

cudaError_t launch_scatter_f64(const DevLattice &L, const double *in, int layout, void *f,
                               cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, scatter_impl, L, in, layout, f, s);
}

namespace {
// Instability check of a stored state (no table): every slot finite, and the
// moments of each site's own slots give rho > 0 and |j|^2 <= u_max^2 rho^2.
// A failing block writes `tag` into *flag if it is still 0, so the flag
// keeps the first failing check of a series.
template <int Q, int HALF>
__global__ void __launch_bounds__(kBlock)
k_stability(const DevLattice L, const typename Store<HALF>::T *__restrict__ f, float u_max2, int tag,
            int *__restrict__ flag) {
    using S = Store<HALF>;
    const int x = blockIdx.x * kBlock + threadIdx.x;
    bool bad = false;
    if (x < L.n) {
        float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
        bool finite = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const float d = S::load(f + (int64_t)i * L.npad + x, L.inv_scale);
            finite = finite && isfinite(d);
            drho += d;
            if (cdir<Q>(i, 0)) jx += cdir<Q>(i, 0) * d;
            if (cdir<Q>(i, 1)) jy += cdir<Q>(i, 1) * d;
            if (cdir<Q>(i, 2)) jz += cdir<Q>(i, 2) * d;
        }
        const float rho = L.rho0 + drho;
        bad = !finite || !(rho > 0.f) || !(jx * jx + jy * jy + jz * jz <= u_max2 * rho * rho);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(flag, 0, tag);
}

// Guard words: the padding slots [n, npad) of every plane and `extra` slots
// after the last plane, set to (fill) or compared with (check) a NaN bit
// pattern; a mismatch sets *flag.
template <typename W>
__global__ void __launch_bounds__(kBlock)
k_guards(W *__restrict__ f, int q, int64_t n, int64_t npad, int64_t extra, W pattern, int check,
         int *__restrict__ flag) {
    const int64_t pad = npad - n;
    const int64_t total = (int64_t)q * pad + extra;
    bool bad = false;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < total; e += (int64_t)gridDim.x * kBlock) {
        const int64_t off = e < (int64_t)q * pad ? (e / pad) * npad + n + e % pad : (int64_t)q * npad + (e - (int64_t)q * pad);
        if (check) bad = bad || f[off] != pattern;
        else f[off] = pattern;
    }
    if (check && __syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

template <int Q, int HALF>
cudaError_t stability_impl(const DevLattice &L, const void *f, float u_max2, int tag, int *flag,
                           cudaStream_t s) {
    k_stability<Q, HALF><<<grid_for(L.n), kBlock, 0, s>>>(L, (const typename Store<HALF>::T *)f, u_max2, tag,
                                                          flag);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_stability(const DevLattice &L, const void *f, float u_max, int tag, int *flag,
                             cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, stability_impl, L, f, u_max * u_max, tag, flag, s);
}

cudaError_t launch_guards(const DevLattice &L, void *f, bool check, int *flag, cudaStream_t s) {
    const int64_t total = (int64_t)L.q * (L.npad - L.n) + kGuardSlots;
    const unsigned g = (unsigned)std::min<int64_t>((total + kBlock - 1) / kBlock, 4 * 152);
    if (L.storage)  // fp16: a NaN pattern; int16: -32768, which no store writes
        k_guards<unsigned short><<<g, kBlock, 0, s>>>((unsigned short *)f, L.q, L.n, L.npad, kGuardSlots,
                                                      (unsigned short)(L.storage == 2 ? 0x8000u : 0x7DA5u),
                                                      check ? 1 : 0, flag);
    else
        k_guards<unsigned><<<g, kBlock, 0, s>>>((unsigned *)f, L.q, L.n, L.npad, kGuardSlots, 0x7FA5A5A5u,
                                                check ? 1 : 0, flag);
    return cudaGetLastError();
}

cudaError_t launch_zero(const DevLattice &L, void *f, cudaStream_t s) {
    const size_t elem = L.storage ? 2 : 4;
    return cudaMemsetAsync(f, 0, elem * (size_t)L.q * (size_t)L.npad, s);
}

}  // namespace hemelb_gb300
