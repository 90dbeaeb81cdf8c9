// Step kernels of libhemelb_gb300 (sm_103a): the fused collide-and-stream
// update of the sparse, Morton-ordered site list in its three forms (pull,
// table-staged persistent pull, AA in place), all built on one collision
// function.
//
// The method (arXiv 1906.11925, Section 2): collision then propagation of a
// single-particle distribution on a sparse lattice of fluid sites, D3Q19
// (Fig. 1); simple bounce-back walls (Section 4).  Collision is LBGK with the
// compressible second-order equilibrium; iolets impose a density through the
// equilibrium populations entering from the iolet (see lbm.h).
//
// Pull storage: the buffer read at step t holds, for every site x and
// direction i, the slot P_i(x) that the pull of step t reads; this is the
// post-collision population f*_i(x, t-1) for fluid and wall links, and for
// an iolet link the equilibrium population already evaluated at the iolet
// density.  Reading the slots through the table (lbm_internal.h) is a
// permutation, so the gather reproduces f(t) exactly.  Values are
// deviations d = f - w_i rho0, in float or in IEEE half scaled by 2^S.
//
// The step is a bandwidth-bound sparse stencil (about one flop per byte): no
// tensor cores.  One site per thread; the q - 1 table entries are coalesced
// (or staged in shared memory by bulk asynchronous copies); the q population
// reads are gathers through the read-only path, made local by the Morton
// order; the q stores are coalesced and streamed.
#include <climits>
#include <cuda_fp16.h>

#include <algorithm>

#include "lattice.h"
#include "lbm_internal.h"
#include "staging.cuh"

namespace hemelb_gb300 {
namespace {

constexpr int kBlock = 256;
// resident blocks per SM requested from the register allocator for the step
// kernel (fp32 storage, fp16 storage)
#ifndef HGB_STEP_MINB_FP32
#define HGB_STEP_MINB_FP32 3
#endif
#ifndef HGB_STEP_MINB_FP16
#define HGB_STEP_MINB_FP16 4
#endif

inline unsigned grid_for(int n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// Raw stored values for the step kernel: fp16 values stay in their scaled
// units (d * 2^S) through the whole update, so that no load or store pays a
// multiplication; only rho and u are formed in real units.
template <int HALF>
struct Raw;  // 0: float, 1: IEEE half, 2: int16 fixed point (both 16-bit forms in units of 2^-S)

// Cache policy of the in-place AA kernels: 1 = evict-first (.cs), 0 = default
#ifndef HGB_AA_LD_CS
#define HGB_AA_LD_CS 0
#endif
#ifndef HGB_AA_ST_CS
#define HGB_AA_ST_CS 1
#endif

template <>
struct Raw<0> {
    using T = float;
    static __device__ __forceinline__ void st_plain(float *p, float v) { *p = v; }
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float ld_cg(const float *p) { return __ldcg(p); }
    static __device__ __forceinline__ float ld_rw(const float *p) { return HGB_AA_LD_CS ? __ldcs(p) : *p; }
    static __device__ __forceinline__ void st(float *p, float v) { __stcs(p, v); }
    static __device__ __forceinline__ void st_rw(float *p, float v) {
        if (HGB_AA_ST_CS) __stcs(p, v);
        else *p = v;
    }
};

template <>
struct Raw<1> {
    using T = __half;
    static __device__ __forceinline__ void st_plain(__half *p, float v) { *p = __float2half_rn(v); }
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float ld_cg(const __half *p) {
        return __half2float(__short_as_half(__ldcg(reinterpret_cast<const short *>(p))));
    }
    static __device__ __forceinline__ float ld_rw(const __half *p) {
        return HGB_AA_LD_CS ? __half2float(__short_as_half(__ldcs(reinterpret_cast<const short *>(p))))
                            : __half2float(*p);
    }
    static __device__ __forceinline__ void st_rw(__half *p, float v) {
        if (HGB_AA_ST_CS) __stcs(reinterpret_cast<short *>(p), __half_as_short(__float2half_rn(v)));
        else *p = __float2half_rn(v);
    }
    static __device__ __forceinline__ void st(__half *p, float v) {
        __stcs(reinterpret_cast<short *>(p), __half_as_short(__float2half_rn(v)));
    }
};

// int16 fixed point (storage 2): the stored value is the deviation times 2^S
// rounded to the nearest integer, |value| <= 32766; 32767 and -32767 are the
// saturation codes an out-of-range value is clamped to (the readers outside
// the step kernels turn them into NaN), -32768 is the guard code.  The
// conversions add and remove 1.5 2^23, which places the integer in the low
// bits of a float (exact for |v| < 2^22): two instructions each way, no
// conversion unit.
__device__ __forceinline__ float i16_to_float(int v) { return __int_as_float(0x4B400000 + v) - 12582912.0f; }
__device__ __forceinline__ short float_to_i16(float v) {
    const float c = fminf(fmaxf(v, -32767.0f), 32767.0f);  // (a NaN becomes -32767)
    return (short)(__float_as_int(c + 12582912.0f) - 0x4B400000);
}
template <>
struct Raw<2> {
    using T = short;
    static __device__ __forceinline__ void st_plain(short *p, float v) { *p = float_to_i16(v); }
    static __device__ __forceinline__ float ld(const short *p) { return i16_to_float(__ldg(p)); }
    static __device__ __forceinline__ float ld_cg(const short *p) { return i16_to_float(__ldcg(p)); }
    static __device__ __forceinline__ float ld_rw(const short *p) {
        return i16_to_float(HGB_AA_LD_CS ? __ldcs(p) : *p);
    }
    static __device__ __forceinline__ void st_rw(short *p, float v) {
        if (HGB_AA_ST_CS) __stcs(p, float_to_i16(v));
        else *p = float_to_i16(v);
    }
    static __device__ __forceinline__ void st(short *p, float v) { __stcs(p, float_to_i16(v)); }
};

// Checked builds (HGB_CHECK_TABLE=1, libhemelb_gb300_checked.so): every table
// entry a step kernel loads is range-checked.  An entry that is none of a
// site index in [0, n), -1 (wall), -2 - k for an iolet k of the lattice or an
// interpolated-wall code sets *L.err = 2 (lbm_mass reports it) and is read as
// a wall link, so that no access leaves the buffers.  No trap.
#ifndef HGB_CHECK_TABLE
#define HGB_CHECK_TABLE 0
#endif
__device__ __forceinline__ int checked_entry(const DevLattice &L, int e) {
    if (!HGB_CHECK_TABLE) return e;
    const bool ok = (e >= 0 && e < L.n) || e == -1 || (e <= -2 && e >= -1 - L.n_iolets) ||
                    (is_bfl(e) && e != INT_MIN);
    if (ok) return e;
    atomicExch(L.err, 2);
    return -1;
}

// Checked builds: a slot-table entry outside the population buffer sets
// *L.err = 2 and is replaced by the site's own slot `own` (the wall link's).
__device__ __forceinline__ unsigned checked_slot(const DevLattice &L, unsigned e, unsigned own) {
    if (!HGB_CHECK_TABLE) return e;
    if (e < (unsigned)L.q * (unsigned)L.npad) return e;
    atomicExch(L.err, 2);
    return own;
}

// Base pointers of the q population planes of one buffer, and of the q - 1
// rows of the slot table, passed by value: an access to plane i of site x is
// then one multiply-add of x onto a pointer held in the constant bank, with
// no per-plane offset to form.
template <typename T>
struct Planes {
    T *p[19];
};
struct SlotRows {
    const uint32_t *p[18];
};

// Velocity moments of one site after its collision (for the iolet values).
struct Velocity {
    float ux, uy, uz, usq15, rs;  // rs: density in stored units
};

// LBGK collision of one site in stored units (deviations, times 2^S for
// fp16), written per opposite pair (i, opp i): with cu = c_i.u the
// equilibrium deviations are sym +- asym, sym = w (drho + rho (4.5 cu^2 -
// 1.5 u^2)), asym = 3 w rho cu, and f*_i = (1 - 1/tau) d_i + (1/tau) deq_i.
//
// The collision conserves mass and momentum, and in float32 it must do so up
// to rounding noise, not up to a constant factor: the products of 1/tau and
// the weights are constants whose rounding errors have the same sign at every
// site and step, so a collision written directly from them scales the
// momentum by about 1 + 1e-8 per step, which adds up coherently (a relative
// error of 1e-4 in u after 5,000 steps).  So the pairs off the axes are
// relaxed as above, and the two conserved quantities fix the rest:
//   axis pair a (directions +a, -a): its sum is relaxed as above, its
//     difference is j_a minus the post-collision momentum of the other pairs
//     along a (the momentum after the collision is the momentum before it);
//   rest population: drho minus the sum of all the others (the mass after
//     the collision is the mass before it).
// In exact arithmetic this is the same collision.
// Every step kernel (pull, AA even, AA odd) uses this one function, so all
// streaming forms give bitwise identical populations.
template <int Q, int HALF>
__device__ __forceinline__ Velocity collide(const DevLattice &L, const float (&d)[Q], float (&out)[Q]) {
    float drs = d[0], jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float sum = d[i] + d[i + 1], dif = d[i] - d[i + 1];
        drs += sum;
        if (cdir<Q>(i, 0)) jx += cdir<Q>(i, 0) * dif;
        if (cdir<Q>(i, 1)) jy += cdir<Q>(i, 1) * dif;
        if (cdir<Q>(i, 2)) jz += cdir<Q>(i, 2) * dif;
    }
    const float rho = HALF ? fmaf(drs, L.inv_scale, L.rho0) : L.rho0 + drs;
    const float ir = (HALF ? L.inv_scale : 1.0f) / rho;
    Velocity v;
    v.ux = jx * ir;
    v.uy = jy * ir;
    v.uz = jz * ir;
    v.usq15 = 1.5f * (v.ux * v.ux + v.uy * v.uy + v.uz * v.uz);
    const float rs = HALF ? rho * L.scale : rho;  // rho in stored units
    v.rs = rs;
    const float om = L.omega, omc = 1.0f - L.omega;
    // pairs off the axes (i >= 7): relaxed towards the equilibrium; their
    // post-collision momentum along each axis and their mass are summed
    float mx = 0.f, my = 0.f, mz = 0.f, mass = 0.f;
#pragma unroll
    for (int i = 7; i < Q; i += 2) {
        const float w = (float)wdir<Q>(i);
        const float cu = cdir<Q>(i, 0) * v.ux + cdir<Q>(i, 1) * v.uy + cdir<Q>(i, 2) * v.uz;
        const float t = fmaf(4.5f * cu, cu, -v.usq15);
        const float sym = fmaf(om * w * rs, t, om * w * drs);
        const float asym = (3.0f * om * w * rs) * cu;
        out[i] = fmaf(omc, d[i], sym + asym);
        out[i + 1] = fmaf(omc, d[i + 1], sym - asym);
        const float m = out[i] - out[i + 1];
        if (cdir<Q>(i, 0)) mx += cdir<Q>(i, 0) * m;
        if (cdir<Q>(i, 1)) my += cdir<Q>(i, 1) * m;
        if (cdir<Q>(i, 2)) mz += cdir<Q>(i, 2) * m;
        mass += out[i] + out[i + 1];
    }
    // axis pairs (i = 1, 3, 5 along x, y, z): relaxed sum, difference from
    // the momentum balance
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int i = 2 * a + 1;
        const float w = (float)wdir<Q>(i);
        const float cu = a == 0 ? v.ux : (a == 1 ? v.uy : v.uz);
        const float t = fmaf(4.5f * cu, cu, -v.usq15);
        const float sym = fmaf(om * w * rs, t, om * w * drs);
        const float sp = fmaf(omc, d[i] + d[i + 1], sym + sym);
        const float dm = (a == 0 ? jx : (a == 1 ? jy : jz)) - (a == 0 ? mx : (a == 1 ? my : mz));
        out[i] = 0.5f * (sp + dm);
        out[i + 1] = 0.5f * (sp - dm);
        mass += out[i] + out[i + 1];
    }
    // rest population from the mass balance
    out[0] = drs - mass;
    return v;
}

// Iolet links of a site with an iolet link (x >= n_bulk): for every i whose
// table entry s[i] = -2 - k marks link opp(i) as iolet k, the slot read back
// as population i at the next step holds
//   density iolet:  the equilibrium at the iolet density and the site's
//                   current velocity (replacing the outgoing f*_opp(i), which
//                   leaves the domain);
//   velocity iolet: the bounced f*_opp(i) plus Ladd's moving-boundary term
//                   6 w_i rho (c_i . u_b), u_b = weight(x) U_k(t) n_k.
template <int Q, int HALF>
__device__ __forceinline__ void iolet_override(const DevLattice &L, int x, const int (&s)[Q],
                                               const Velocity &v, const IoletStep &io,
                                               const double *__restrict__ rho_io,
                                               const IoletStep *__restrict__ io_dev, float (&out)[Q]) {
    // the step's iolet values: io (a kernel parameter), or the same record in
    // device memory when io_dev is set (the steps of a CUDA graph)
    const unsigned long long vel_mask = io_dev ? io_dev->vel_mask : io.vel_mask;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (s[i] <= -2 && !is_bfl(s[i])) {
            const int k = -2 - s[i];
            float drk, rk;
            if (rho_io) {
                const double r = rho_io[k];
                drk = (float)(r - (double)L.rho0);
                rk = (float)r;
            } else if (io_dev) {
                drk = io_dev->drho[k];
                rk = io_dev->rho[k];
            } else {
                drk = io.drho[k];
                rk = io.rho[k];
            }
            if ((vel_mask >> k) & 1ull) {
                // rk is the speed U_k(t)
                const float *nk = io_dev ? io_dev->nrm[k] : io.nrm[k];
                const float wu = L.vel_weight[x - L.n_bulk] * rk;
                const float cn = cdir<Q>(i, 0) * nk[0] + cdir<Q>(i, 1) * nk[1] + cdir<Q>(i, 2) * nk[2];
                out[opp(i)] += 6.0f * (float)wdir<Q>(i) * v.rs * wu * cn;
                continue;
            }
            if (HALF) {
                drk *= L.scale;
                rk *= L.scale;
            }
            const float cu = cdir<Q>(i, 0) * v.ux + cdir<Q>(i, 1) * v.uy + cdir<Q>(i, 2) * v.uz;
            out[opp(i)] = (float)wdir<Q>(i) * (drk + rk * (3.0f * cu + 4.5f * cu * cu - v.usq15));
        }
    }
}

// Interpolated (BFL) walls (entries is_bfl(s[p]): link opp(p) is a wall at
// fluid fraction q; the population p of the next step is read back from the
// site's own slot, the slot that holds out[opp(p)] after the step in every
// streaming form: pull slot opp(p), AA even slot p, AA odd own slot p).  The
// gathered d[] and the collision's out[] mean the same in every form, so the
// same two helpers serve the pull and the AA kernels.
//   bfl_gather:  q < 1/2 with a fluid upstream site (s[opp(p)] >= 0): the
//                slot holds 2q f*_opp(p)(x); add (1 - 2q) f*_opp(p)(x - c_opp(p)),
//                the population opp(p) just pulled from the upstream site;
//   bfl_scatter: after the collision, the slot opp(p) receives 2q f*_opp(p)
//                (q < 1/2, fluid upstream), f*_opp(p) (q < 1/2, no fluid
//                upstream: half-way rule), or f*_opp(p)/(2q) + (1 - 1/(2q)) f*_p
//                (q >= 1/2), all from the collision's own values.
template <int Q>
__device__ __forceinline__ void bfl_gather(const int (&s)[Q], float (&d)[Q]) {
#pragma unroll
    for (int p = 1; p < Q; ++p) {
        if (is_bfl(s[p])) {
            const float qv = bfl_q(s[p]);
            if (qv < 0.5f && s[opp(p)] >= 0) d[p] = fmaf(1.0f - 2.0f * qv, d[opp(p)], d[p]);
        }
    }
}

template <int Q>
__device__ __forceinline__ void bfl_scatter(const int (&s)[Q], float (&out)[Q]) {
#pragma unroll
    for (int a = 1; a < Q; a += 2) {
        const int b = a + 1;  // opp(a)
        const float ra = out[a], rb = out[b];
        if (is_bfl(s[b])) {  // wall along c_a: slot a feeds population b
            const float qv = bfl_q(s[b]);
            if (qv < 0.5f) {
                if (s[a] >= 0) out[a] = 2.0f * qv * ra;
            } else {
                const float h = 0.5f / qv;
                out[a] = fmaf(h, ra, (1.0f - h) * rb);
            }
        }
        if (is_bfl(s[a])) {  // wall along c_b: slot b feeds population a
            const float qv = bfl_q(s[a]);
            if (qv < 0.5f) {
                if (s[b] >= 0) out[b] = 2.0f * qv * rb;
            } else {
                const float h = 0.5f / qv;
                out[b] = fmaf(h, rb, (1.0f - h) * ra);
            }
        }
    }
}

// Fused pull collide-and-stream of one time step, one site per thread.
//   gather   d_i = slot(i, x) through the table (coalesced table reads,
//            gathered population reads, Morton order keeps them local);
//   collide  collide() above;
//   iolets   sites with iolet links come last in the internal order
//            (x >= n_bulk): iolet_override() above;
//   stream   q coalesced streaming stores at the site's own slots.
// All slot offsets are 32-bit (q * npad < 2^31 is checked at create).
// IO = false: the bulk sites [0, n_bulk); IO = true: the sites with an
// iolet link [n_bulk, n), launched separately so that the bulk kernel carries
// no iolet code (and no register cost for it).
// resident blocks per SM for the launch of the sites with iolet or
// interpolated-wall links
#ifndef HGB_TAIL_MINB_FP32
#define HGB_TAIL_MINB_FP32 4
#endif
#ifndef HGB_TAIL_MINB_FP16
#define HGB_TAIL_MINB_FP16 HGB_STEP_MINB_FP16
#endif
template <int Q, int HALF, bool IO, bool BFL = false>
__global__ void __launch_bounds__(kBlock, IO ? (HALF ? HGB_TAIL_MINB_FP16 : HGB_TAIL_MINB_FP32)
                                             : (HALF ? HGB_STEP_MINB_FP16 : HGB_STEP_MINB_FP32))
k_step(const DevLattice L, const typename Raw<HALF>::T *__restrict__ fin,
       typename Raw<HALF>::T *__restrict__ fout, const Planes<typename Raw<HALF>::T> OP, const SlotRows S,
       const IoletStep io, const double *__restrict__ rho_io, const IoletStep *__restrict__ io_dev) {
    using R = Raw<HALF>;
    const int x = (IO ? L.n_bulk : 0) + blockIdx.x * kBlock + threadIdx.x;
    if (x >= (IO ? L.n : L.n_bulk)) return;
    const unsigned np = (unsigned)L.npad;
    if constexpr (!IO && !BFL) {
        // bulk sites: gather through the slot table, store through the planes
        float d[Q], out[Q];
        d[0] = R::ld(fin + x);
#pragma unroll
        for (int i = 1; i < Q; ++i)
            d[i] = R::ld(fin + checked_slot(L, __ldcs(S.p[i - 1] + x), (unsigned)opp(i) * np + (unsigned)x));
        collide<Q, HALF>(L, d, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) R::st(OP.p[i] + x, out[i]);
    } else {
        int s[Q];
#pragma unroll
        for (int i = 1; i < Q; ++i) s[i] = checked_entry(L, __ldcs(L.tab + (unsigned)(i - 1) * np + (unsigned)x));
        float d[Q];
        d[0] = R::ld(fin + x);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const unsigned e = s[i] >= 0 ? (unsigned)i * np + (unsigned)s[i]
                                         : (unsigned)opp(i) * np + (unsigned)x;
            d[i] = R::ld(fin + e);
        }
        if (BFL) bfl_gather<Q>(s, d);
        float out[Q];
        const Velocity v = collide<Q, HALF>(L, d, out);
        if (BFL) bfl_scatter<Q>(s, out);
        if (IO) iolet_override<Q, HALF>(L, x, s, v, io, rho_io, io_dev, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) R::st(fout + (unsigned)i * np + (unsigned)x, out[i]);
    }
}

// ---------------------------------------------------------------------------
// Table-staged persistent variant of the pull step (bulk sites only).  Each
// CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...; one thread
// copies the q - 1 table rows of a tile (256 int32 each) into shared memory
// with bulk asynchronous copies completing on an mbarrier, two tiles ahead,
// so the table reads leave the threads' load path and arrive while the
// previous tile computes.  Every wait is bounded: on a timeout the CTA sets
// *err, waits (bounded) for its other copy in flight, and returns.  The copy
// it gave up on may still land later, in shared memory that another CTA then
// owns, so after a give-up the whole output of the launch is undefined:
// lbm_mass reports the flag and the context refuses to step until its state
// is replaced (lbm_set_state, lbm_set_populations).
#ifndef HGB_STEP_STAGED
#define HGB_STEP_STAGED 1
#endif
#ifndef HGB_STAGES
#define HGB_STAGES 2
#endif
// persistent CTAs per SM of the staged kernel (0: as many as fit)
#ifndef HGB_STAGED_CTAS
#define HGB_STAGED_CTAS 0
#endif
constexpr int kStages = HGB_STAGES;

template <int Q, int HALF>
__global__ void __launch_bounds__(kBlock, HALF ? HGB_STEP_MINB_FP16 : HGB_STEP_MINB_FP32)
k_step_staged(const DevLattice L, const typename Raw<HALF>::T *__restrict__ fin,
              const Planes<typename Raw<HALF>::T> out_planes, int *__restrict__ err) {
    using R = Raw<HALF>;
    constexpr int NE = Q - 1;
    constexpr int SB = NE * kTile * 4;
    static_assert(kBlock == kTile, "one site per thread per tile");
    extern __shared__ __align__(128) unsigned char sbuf[];  // [kStages][SB]
    __shared__ __align__(8) uint64_t bar[kStages];
    __shared__ int ok;
    const int tid = threadIdx.x;
    const int ntiles = (L.n_bulk + kBlock - 1) / kBlock;
    const unsigned np = (unsigned)L.npad;
    auto issue = [&](int stage, int tile) {
        unsigned char *dst = sbuf + stage * SB;
        // ragged last tile: round the row up to 16 bytes (stays inside the
        // plane: npad is a multiple of 128 and >= n_bulk)
        const int count = min(kBlock, L.n_bulk - tile * kBlock);
        const unsigned bytes = ((unsigned)count * 4u + 15u) & ~15u;
        mbar_expect_tx(&bar[stage], bytes * NE);
#pragma unroll 1
        for (int i = 0; i < NE; ++i)
            bulk_g2s(dst + i * kBlock * 4, L.slots + (size_t)i * np + (size_t)tile * kBlock, bytes, &bar[stage]);
    };
    if (tid == 0) {
        for (int st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        for (int st = 0; st < kStages; ++st) {
            const int tile = blockIdx.x + st * gridDim.x;
            if (tile < ntiles) issue(st, tile);
        }
    }
    __syncthreads();
    int k = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
        const int stage = k % kStages;
        const unsigned parity = (unsigned)(k / kStages) & 1u;
        if (tid == 0) ok = mbar_wait_bounded(&bar[stage], parity) ? 1 : 0;
        __syncthreads();
        if (!ok) {
            if (tid == 0) {
                atomicExch(err, 1);
                // the other stage's copy, if one is in flight
                const int other = tile + gridDim.x;
                if (other < ntiles) mbar_wait_bounded(&bar[(k + 1) % kStages], (unsigned)((k + 1) / kStages) & 1u);
            }
            return;
        }
        const int x = tile * kBlock + tid;
        // (the rows of a ragged last tile run past n_bulk: only the tile's
        // sites read them)
        if (x < L.n_bulk) {
            const uint32_t *rows = reinterpret_cast<const uint32_t *>(sbuf + stage * SB);
            float d[Q];
            d[0] = R::ld(fin + x);
#pragma unroll
            for (int i = 1; i < Q; ++i)
                d[i] = R::ld(fin + checked_slot(L, rows[(i - 1) * kTile + tid], (unsigned)opp(i) * np + (unsigned)x));
            float out[Q];
            collide<Q, HALF>(L, d, out);
#pragma unroll
            for (int i = 0; i < Q; ++i) R::st(out_planes.p[i] + x, out[i]);
        }
        __syncthreads();  // every thread is done with this stage's buffer
        if (tid == 0) {
            const int nt = tile + kStages * gridDim.x;
            if (nt < ntiles) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(stage, nt);
            }
        }
    }
}

// resident blocks per SM of the AA step kernels (fp32, 16-bit storage)
#ifndef HGB_AA_MINB_FP32
#define HGB_AA_MINB_FP32 4
#endif
#ifndef HGB_AA_MINB_FP16
#define HGB_AA_MINB_FP16 4
#endif

// The plane length, read afresh where it is used: inside the fused pair's
// persistent loop the compiler would otherwise keep the q plane offsets
// i * npad live across the whole loop (loop-invariant), which costs the
// registers the bodies need.
__device__ __forceinline__ unsigned fresh_npad(const DevLattice &L) {
    unsigned v;
    asm volatile("mov.u32 %0, %1;" : "=r"(v) : "r"((unsigned)L.npad));
    return v;
}

// The bulk-site bodies of the AA step (shared by k_step_aa and the fused step
// pair below, so that both give the same bits).  Even step: the site's own
// slots (measured: fp16 is faster through the plane pointers, each address
// one multiply-add onto a pointer in the constant bank, formed again for the
// store; fp32 through one base pointer and the plane offsets).  Odd step:
// through the slot table.  FUSED: the body runs inside the fused step pair,
// where other blocks of the same launch wrote the slots it reads: loads
// bypass L1 (.cg), so that no line cached before the write is read, and the
// even step's stores keep their lines in L2 for the odd step (default policy
// instead of evict-first).
template <int Q, int HALF, bool FUSED>
__device__ __forceinline__ void aa_even_bulk(const DevLattice &L, typename Raw<HALF>::T *__restrict__ A,
                                             const Planes<typename Raw<HALF>::T> &P, int x) {
    using R = Raw<HALF>;
    const unsigned np = FUSED ? fresh_npad(L) : (unsigned)L.npad;
    float d[Q], out[Q];
    if (HALF && !FUSED) {
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = R::ld_rw(P.p[i] + x);
        collide<Q, HALF>(L, d, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) R::st_rw(P.p[i] + x, out[opp(i)]);
    } else {
        typename Raw<HALF>::T *a = A + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = FUSED ? R::ld_cg(a + (unsigned)i * np) : R::ld_rw(a + (unsigned)i * np);
        collide<Q, HALF>(L, d, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (FUSED) R::st_plain(a + (unsigned)i * np, out[opp(i)]);
            else R::st_rw(a + (unsigned)i * np, out[opp(i)]);
        }
    }
}

template <int Q, int HALF, bool FUSED>
__device__ __forceinline__ void aa_odd_bulk(const DevLattice &L, typename Raw<HALF>::T *__restrict__ A,
                                            const SlotRows &S, int x) {
    using R = Raw<HALF>;
    const unsigned np = FUSED ? fresh_npad(L) : (unsigned)L.npad;
    float d[Q], out[Q];
    unsigned e[Q];
    e[0] = (unsigned)x;
    const uint32_t *srow = L.slots + x;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        e[i] = checked_slot(L, __ldcs(FUSED ? srow + (unsigned)(i - 1) * np : S.p[i - 1] + x),
                            (unsigned)i * np + (unsigned)x);
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = FUSED ? R::ld_cg(A + e[i]) : R::ld_rw(A + e[i]);
    collide<Q, HALF>(L, d, out);
#pragma unroll
    for (int i = 0; i < Q; ++i) R::st_rw(A + e[i], out[opp(i)]);
}

// Bounded wait of the fused step pair for a counter that other blocks of the
// same launch raise: polls (acquire, GPU scope) at most `limit` times with a
// short sleep between polls, about a second in all; false if it gave up.
constexpr unsigned kPairSpinLimit = 1u << 21;
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ bool wait_count(const unsigned *p, unsigned need, unsigned limit = kPairSpinLimit) {
    for (unsigned it = 0; it < limit; ++it) {
        if (ld_acquire(p) >= need) return true;
        __nanosleep(64);
    }
    return false;
}
// The same for the three chunks c - 1 .. c + 1 at once, by warp 0 (lane l
// polls chunk c - 1 + l; called by all 32 lanes).
__device__ __forceinline__ bool wait_chunks(const unsigned *done, const int *tiles, int c, int nchunks, int lane) {
    const int cc = c - 1 + lane;
    const bool mine = lane < 3 && cc >= 0 && cc < nchunks;
    const unsigned need = mine ? (unsigned)tiles[cc] : 0u;
    for (unsigned it = 0; it < kPairSpinLimit; ++it) {
        const unsigned v = mine ? ld_acquire(done + cc) : 0u;
        if (__all_sync(0xffffffffu, v >= need)) return true;
        __nanosleep(64);
    }
    return false;
}

// The two bounded waits, checked on their own (lbm_check_wait_timeout): the
// staged kernels' mbarrier wait on a barrier that expects 16 bytes no copy
// will ever deliver (bit 0 of *err when it gives up), and the fused step
// pair's counter wait on a counter nothing raises (bit 1).  No copy is
// issued, so nothing is in flight when the kernel returns.
__global__ void k_wait_probe(int *err, const unsigned *never, unsigned limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16u);
    if (!mbar_wait_bounded(&bar, 0u, limit)) atomicOr(err, 1);
    if (!wait_count(never, 1u, limit)) atomicOr(err, 2);
}

// A fused AA step pair (LBM_ORDER_SLABS): one persistent launch works through
// the plan's items in list order, each block taking the next item from a
// counter.  An even run writes only its own sites' slots and, once its block
// is done, counts itself done for its chunk (release); an odd run of chunk c
// reads and writes slots of the chunks c - 1 .. c + 1 only, so it first waits
// (acquire) until their even runs are all done.  The runs it waits for come
// earlier in the list and were taken by blocks that are running, so every
// wait ends.  The two steps of one chunk are a fixed number of chunks apart
// in the list (the host's lag), so the odd step reads the even step's output
// back from L2.  A wait that gives
// up sets *err and the block stops taking items (the state is then partly
// updated and the host refuses further steps).  The last block to finish
// clears the counters for the next launch.
#ifndef HGB_AA_PAIR_MINB
#define HGB_AA_PAIR_MINB 4
#endif
template <int Q, int HALF>
__global__ void __launch_bounds__(kBlock, HGB_AA_PAIR_MINB)
k_step_aa_pair(const DevLattice L, typename Raw<HALF>::T *__restrict__ A, const Planes<typename Raw<HALF>::T> P,
               const SlotRows S, const PairPlan W, int *__restrict__ err) {
    __shared__ int item, ok;
    const int tid = (int)threadIdx.x;
    unsigned *next = W.ctr, *finished = W.ctr + 1, *done = W.ctr + 2;
    bool failed = false;
    for (;;) {
        if (tid == 0) item = (int)atomicAdd(next, 1u);
        __syncthreads();
        const int it = item;
        if (it >= W.n_items) break;
        const int4 w = W.items[it];
        const int x = w.x + tid;
        if (w.w) {
            if (tid < 32) {
                const bool good = wait_chunks(done, W.tiles, w.z, W.nchunks, tid);
                if (tid == 0) ok = good ? 1 : 0;
            }
            __syncthreads();
            if (!ok) {
                failed = true;
                break;
            }
            if (x < w.y) aa_odd_bulk<Q, HALF, true>(L, A, S, x);
        } else {
            if (x < w.y) aa_even_bulk<Q, HALF, true>(L, A, P, x);
            __syncthreads();
            if (tid == 0) {
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                atomicAdd(done + w.z, 1u);
            }
        }
        __syncthreads();  // every thread has read `item` and `ok`
    }
    if (tid == 0) {
        if (failed) atomicExch(err, 1);
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (atomicAdd(finished, 1u) == gridDim.x - 1) {
            for (int c = 0; c < W.nchunks; ++c) done[c] = 0u;
            *next = 0u;
            *finished = 0u;
        }
    }
}

// AA-pattern in-place step on one population buffer A (Bailey et al.,
// "Accelerating lattice Boltzmann fluid flow simulations using graphics
// processors", ICPP 2009).  Population i of site x is read from its slot and
// the post-collision population opp(i) is written back into that same slot,
// so every slot is read and written by one thread only:
//   even step: slot_i = A[i][x]                  (own site, no table for bulk sites)
//   odd step:  slot_i = A[opp(i)][x - c_i]       (through the table), or
//              A[i][x] for a wall or iolet link opp(i).
// The bulk sites (IO = false) take the plane pointers P for the even step and
// the slot table rows S (DevLattice::slots, these very slot_i) for the odd
// step; the sites with iolet links decode the pull table.
// After an even step A holds the populations of time t+1 in swapped slots;
// after an odd step they are back in natural order, A[i][x] = f_i(x).
// the even bulk step (no table) on its own
#ifndef HGB_AA_MINB_EVEN_FP32
#define HGB_AA_MINB_EVEN_FP32 HGB_AA_MINB_FP32
#endif
#ifndef HGB_AA_MINB_EVEN_FP16
#define HGB_AA_MINB_EVEN_FP16 HGB_AA_MINB_FP16
#endif
template <int Q, int HALF, bool ODD, bool IO, bool BFL = false>
__global__ void __launch_bounds__(kBlock, (ODD || IO) ? (HALF ? HGB_AA_MINB_FP16 : HGB_AA_MINB_FP32)
                                                      : (HALF ? HGB_AA_MINB_EVEN_FP16 : HGB_AA_MINB_EVEN_FP32))
k_step_aa(const DevLattice L, typename Raw<HALF>::T *__restrict__ A, const Planes<typename Raw<HALF>::T> P,
          const SlotRows S, const IoletStep io, const double *__restrict__ rho_io,
          const IoletStep *__restrict__ io_dev) {
    using R = Raw<HALF>;
    const int x = (IO ? L.n_bulk : 0) + blockIdx.x * kBlock + threadIdx.x;
    if (x >= (IO ? L.n : L.n_bulk)) return;
    const unsigned np = (unsigned)L.npad;
    float d[Q];
    float out[Q];
    if (!IO) {
        // bulk sites: even step on the own slots through the plane pointers,
        // odd step through the slot table; no table codes, no iolet work
        if (HGB_PF_BLOCKS > 0) {
            // the population rows (and, for the odd step, the slot-table
            // rows) of the tile HGB_PF_BLOCKS blocks ahead
            const unsigned x0 = (blockIdx.x + HGB_PF_BLOCKS) * (unsigned)kBlock;
            const int r = (int)threadIdx.x;
            prefetch_rows(A, sizeof(typename Raw<HALF>::T), np, Q, x0, (unsigned)L.n_bulk, np, r);
            if (ODD) prefetch_rows(L.slots, 4u, np, Q - 1, x0, (unsigned)L.n_bulk, np, r - Q);
        }
        if (!ODD)
            aa_even_bulk<Q, HALF, false>(L, A, P, x);
        else
            aa_odd_bulk<Q, HALF, false>(L, A, S, x);
        return;
    }
    int s[Q];
    s[0] = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i) s[i] = checked_entry(L, __ldcs(L.tab + (unsigned)(i - 1) * np + (unsigned)x));
    if (!ODD) {
        // own slots: one base pointer, plane stride np
        typename Raw<HALF>::T *a = A + x;
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = R::ld_rw(a + (unsigned)i * np);
        if (BFL) bfl_gather<Q>(s, d);
        const Velocity v = collide<Q, HALF>(L, d, out);
        if (BFL) bfl_scatter<Q>(s, out);
        if (IO) iolet_override<Q, HALF>(L, x, s, v, io, rho_io, io_dev, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) R::st_rw(a + (unsigned)i * np, out[opp(i)]);
    } else {
        // slot of population i (32-bit element offset)
        auto slot = [&](int i) -> unsigned {
            if (i == 0) return (unsigned)x;
            return s[i] >= 0 ? (unsigned)opp(i) * np + (unsigned)s[i] : (unsigned)i * np + (unsigned)x;
        };
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = R::ld_rw(A + slot(i));
        if (BFL) bfl_gather<Q>(s, d);
        const Velocity v = collide<Q, HALF>(L, d, out);
        if (BFL) bfl_scatter<Q>(s, out);
        if (IO) iolet_override<Q, HALF>(L, x, s, v, io, rho_io, io_dev, out);
#pragma unroll
        for (int i = 0; i < Q; ++i) R::st_rw(A + slot(i), out[opp(i)]);
    }
}

// The AA step out of place, from the state in S into D (the same slots as
// k_step_aa reads and writes, S and D distinct; every slot of D is written):
// the first step of a recomputation from an adjoint snapshot, which must stay
// intact.  The per-site arithmetic is k_step_aa's.
template <int Q, int HALF, bool ODD, bool IO, bool BFL = false>
__global__ void __launch_bounds__(kBlock, HALF ? HGB_AA_MINB_FP16 : HGB_AA_MINB_FP32)
k_step_aa_oop(const DevLattice L, const typename Raw<HALF>::T *__restrict__ S, typename Raw<HALF>::T *__restrict__ D,
              const IoletStep io) {
    using R = Raw<HALF>;
    const int x = (IO ? L.n_bulk : 0) + blockIdx.x * kBlock + threadIdx.x;
    if (x >= (IO ? L.n : L.n_bulk)) return;
    const unsigned np = (unsigned)L.npad;
    int s[Q];
    s[0] = 0;
    if (ODD || IO) {
#pragma unroll
        for (int i = 1; i < Q; ++i) s[i] = __ldg(L.tab + (unsigned)(i - 1) * np + (unsigned)x);
    }
    auto slot = [&](int i) -> unsigned {
        if (!ODD || i == 0) return (unsigned)i * np + (unsigned)x;
        return s[i] >= 0 ? (unsigned)opp(i) * np + (unsigned)s[i] : (unsigned)i * np + (unsigned)x;
    };
    float d[Q], out[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = R::ld(S + slot(i));
    if (BFL) bfl_gather<Q>(s, d);
    const Velocity v = collide<Q, HALF>(L, d, out);
    if (BFL) bfl_scatter<Q>(s, out);
    if (IO) iolet_override<Q, HALF>(L, x, s, v, io, nullptr, nullptr, out);
#pragma unroll
    for (int i = 0; i < Q; ++i) R::st(D + slot(i), out[opp(i)]);
}

// Fork the side stream off s before the bulk launch; returns the stream the
// launch of the sites after the bulk goes to.
inline cudaStream_t fork_side(cudaStream_t s, const SideStream *side, bool both) {
    if (!side || !both) return s;
    if (cudaEventRecord(side->fork, s) != cudaSuccess) return s;
    if (cudaStreamWaitEvent(side->s, side->fork, 0) != cudaSuccess) return s;
    return side->s;
}
inline cudaError_t join_side(cudaStream_t s, cudaStream_t t, const SideStream *side) {
    if (t == s) return cudaSuccess;
    cudaError_t e = cudaEventRecord(side->join, t);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, side->join, 0);
    return e;
}

template <typename T>
Planes<T> planes_of(T *A, int q, int64_t npad) {
    Planes<T> P{};
    for (int i = 0; i < q; ++i) P.p[i] = A + (size_t)i * (size_t)npad;
    return P;
}
inline SlotRows slot_rows_of(const DevLattice &L) {
    SlotRows S{};
    for (int i = 0; i + 1 < L.q; ++i) S.p[i] = L.slots + (size_t)i * (size_t)L.npad;
    return S;
}

template <int Q, int HALF>
cudaError_t step_aa_impl(const DevLattice &L, void *A, bool odd, const IoletStep &io,
                         const double *rho_io, cudaStream_t s, const SideStream *side,
                         const IoletStep *io_dev) {
    using T = typename Raw<HALF>::T;
    const int nb = L.n_bulk, ni = L.n - L.n_bulk;
    const cudaStream_t t = fork_side(s, side, nb > 0 && ni > 0);
    const Planes<T> P = planes_of((T *)A, Q, L.npad);
    const SlotRows S = slot_rows_of(L);
    if (odd) {
        if (nb) k_step_aa<Q, HALF, true, false><<<grid_for(nb), kBlock, 0, s>>>(L, (T *)A, P, S, io, rho_io, io_dev);
        if (ni && L.bfl)
            k_step_aa<Q, HALF, true, true, true><<<grid_for(ni), kBlock, 0, t>>>(L, (T *)A, P, S, io, rho_io, io_dev);
        else if (ni)
            k_step_aa<Q, HALF, true, true><<<grid_for(ni), kBlock, 0, t>>>(L, (T *)A, P, S, io, rho_io, io_dev);
    } else {
        if (nb) k_step_aa<Q, HALF, false, false><<<grid_for(nb), kBlock, 0, s>>>(L, (T *)A, P, S, io, rho_io, io_dev);
        if (ni && L.bfl)
            k_step_aa<Q, HALF, false, true, true><<<grid_for(ni), kBlock, 0, t>>>(L, (T *)A, P, S, io, rho_io, io_dev);
        else if (ni)
            k_step_aa<Q, HALF, false, true><<<grid_for(ni), kBlock, 0, t>>>(L, (T *)A, P, S, io, rho_io, io_dev);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = join_side(s, t, side);
    return e;
}

// An even step and the following odd step of the AA form in one pass: the
// iolet-site even step first, then the persistent fused kernel over the bulk
// sites, then the iolet-site odd step (which reads slots of bulk sites
// anywhere, so it waits for every even step).
template <int Q, int HALF>
int aa_pair_grid(int n_items) {
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_aa_pair<Q, HALF>, kBlock, 0) != cudaSuccess)
            return -1;
        g = sms * std::max(per, 1);
    }
    return std::max(1, std::min(g, n_items));
}

template <int Q, int HALF>
cudaError_t step_aa_pair_impl(const DevLattice &L, void *A, const IoletStep &io_even, const IoletStep &io_odd,
                              cudaStream_t s, const IoletStep *io_dev_even, const IoletStep *io_dev_odd,
                              const PairPlan &W) {
    using T = typename Raw<HALF>::T;
    const int ni = L.n - L.n_bulk;
    const Planes<T> P = planes_of((T *)A, Q, L.npad);
    const SlotRows S = slot_rows_of(L);
    if (!L.err || !W.items || !W.ctr) return cudaErrorInvalidValue;
    if (ni && L.bfl)
        k_step_aa<Q, HALF, false, true, true><<<grid_for(ni), kBlock, 0, s>>>(L, (T *)A, P, S, io_even, nullptr,
                                                                               io_dev_even);
    else if (ni)
        k_step_aa<Q, HALF, false, true><<<grid_for(ni), kBlock, 0, s>>>(L, (T *)A, P, S, io_even, nullptr,
                                                                         io_dev_even);
    if (W.n_items) {
        const int grid = aa_pair_grid<Q, HALF>(W.n_items);
        if (grid < 0) return cudaErrorInvalidConfiguration;
        k_step_aa_pair<Q, HALF><<<grid, kBlock, 0, s>>>(L, (T *)A, P, S, W, L.err);
    }
    if (ni && L.bfl)
        k_step_aa<Q, HALF, true, true, true><<<grid_for(ni), kBlock, 0, s>>>(L, (T *)A, P, S, io_odd, nullptr,
                                                                              io_dev_odd);
    else if (ni)
        k_step_aa<Q, HALF, true, true><<<grid_for(ni), kBlock, 0, s>>>(L, (T *)A, P, S, io_odd, nullptr,
                                                                        io_dev_odd);
    return cudaGetLastError();
}

template <int Q, int HALF>
cudaError_t step_impl(const DevLattice &L, const void *fin, void *fout, const IoletStep &io,
                      const double *rho_io, cudaStream_t s, const SideStream *side,
                      const IoletStep *io_dev) {
    using T = typename Raw<HALF>::T;
    const int nb = L.n_bulk, ni = L.n - L.n_bulk;
    const cudaStream_t t = fork_side(s, side, nb > 0 && ni > 0);
    const Planes<T> OP = planes_of((T *)fout, Q, L.npad);
    const SlotRows S = slot_rows_of(L);
    if (nb) {
        // (measured with the slot table: the staged kernel is faster for 16-bit
        // storage, the plain one for fp32, 354 against 378 us per tree step)
        if (HGB_STEP_STAGED && HALF && L.err) {
            static int grid_cache[2] = {0, 0};
            const size_t smem = (size_t)kStages * (Q - 1) * kTile * 4;
            int &g = grid_cache[HALF ? 1 : 0];
            if (g == 0) {
                int dev = 0, sms = 0, per = 0;
                cudaGetDevice(&dev);
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
                if (smem > 48 * 1024) {
                    cudaError_t e = cudaFuncSetAttribute(k_step_staged<Q, HALF>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                    if (e != cudaSuccess) return e;
                }
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_step_staged<Q, HALF>, kBlock, smem);
                if (HGB_STAGED_CTAS > 0) per = std::min(per, HGB_STAGED_CTAS);
                g = std::max(1, sms * std::max(per, 1));
            }
            const int grid = std::min(g, (nb + kBlock - 1) / kBlock);
            k_step_staged<Q, HALF><<<grid, kBlock, smem, s>>>(L, (const T *)fin, OP, L.err);
        } else {
            k_step<Q, HALF, false><<<grid_for(nb), kBlock, 0, s>>>(L, (const T *)fin, (T *)fout, OP, S, io, rho_io,
                                                                   io_dev);
        }
    }
    if (ni && L.bfl)
        k_step<Q, HALF, true, true><<<grid_for(ni), kBlock, 0, t>>>(L, (const T *)fin, (T *)fout, OP, S, io, rho_io,
                                                                    io_dev);
    else if (ni)
        k_step<Q, HALF, true><<<grid_for(ni), kBlock, 0, t>>>(L, (const T *)fin, (T *)fout, OP, S, io, rho_io,
                                                              io_dev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = join_side(s, t, side);
    return e;
}

}  // namespace

#define HGB_DISPATCH(L, FN, ...)                                                         \
    ((L).q == 15 ? ((L).storage == 2 ? FN<15, 2>(__VA_ARGS__)                                 \
                                     : (L).storage ? FN<15, 1>(__VA_ARGS__) : FN<15, 0>(__VA_ARGS__)) \
                 : ((L).storage == 2 ? FN<19, 2>(__VA_ARGS__)                                 \
                                     : (L).storage ? FN<19, 1>(__VA_ARGS__) : FN<19, 0>(__VA_ARGS__)))

cudaError_t launch_step(const DevLattice &L, const void *fin, void *fout, const IoletStep &io,
                        const double *rho_io, cudaStream_t s, const SideStream *side,
                        const IoletStep *io_dev) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, step_impl, L, fin, fout, io, rho_io, s, side, io_dev);
}

namespace {
template <int Q, int HALF>
cudaError_t step_aa_oop_impl(const DevLattice &L, const void *src, void *dst, bool odd, const IoletStep &io,
                             cudaStream_t s) {
    using T = typename Raw<HALF>::T;
    const int nb = L.n_bulk, ni = L.n - L.n_bulk;
    if (odd) {
        if (nb) k_step_aa_oop<Q, HALF, true, false><<<grid_for(nb), kBlock, 0, s>>>(L, (const T *)src, (T *)dst, io);
        if (ni && L.bfl)
            k_step_aa_oop<Q, HALF, true, true, true><<<grid_for(ni), kBlock, 0, s>>>(L, (const T *)src, (T *)dst, io);
        else if (ni)
            k_step_aa_oop<Q, HALF, true, true><<<grid_for(ni), kBlock, 0, s>>>(L, (const T *)src, (T *)dst, io);
    } else {
        if (nb) k_step_aa_oop<Q, HALF, false, false><<<grid_for(nb), kBlock, 0, s>>>(L, (const T *)src, (T *)dst, io);
        if (ni && L.bfl)
            k_step_aa_oop<Q, HALF, false, true, true><<<grid_for(ni), kBlock, 0, s>>>(L, (const T *)src, (T *)dst,
                                                                                     io);
        else if (ni)
            k_step_aa_oop<Q, HALF, false, true><<<grid_for(ni), kBlock, 0, s>>>(L, (const T *)src, (T *)dst, io);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_step_aa_oop(const DevLattice &L, const void *src, void *dst, bool odd, const IoletStep &io,
                               cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, step_aa_oop_impl, L, src, dst, odd, io, s);
}

cudaError_t launch_step_aa_pair(const DevLattice &L, void *A, const IoletStep &io_even, const IoletStep &io_odd,
                                cudaStream_t s, const IoletStep *io_dev_even, const IoletStep *io_dev_odd,
                                const PairPlan &W) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, step_aa_pair_impl, L, A, io_even, io_odd, s, io_dev_even, io_dev_odd, W);
}

cudaError_t launch_wait_probe(unsigned limit, int *err, const unsigned *never, cudaStream_t s) {
    k_wait_probe<<<1, 32, 0, s>>>(err, never, limit);
    return cudaGetLastError();
}

cudaError_t launch_step_aa(const DevLattice &L, void *A, bool odd, const IoletStep &io,
                           const double *rho_io, cudaStream_t s, const SideStream *side,
                           const IoletStep *io_dev) {
    if (L.n == 0) return cudaSuccess;
    return HGB_DISPATCH(L, step_aa_impl, L, A, odd, io, rho_io, s, side, io_dev);
}

}  // namespace hemelb_gb300
