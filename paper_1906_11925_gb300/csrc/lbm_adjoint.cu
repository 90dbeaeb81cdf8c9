// Discrete adjoint (reverse mode) of the fused collide-and-stream step, for
// gradients of time-windowed objectives with respect to the relaxation time
// and the iolet density schedules.
//
// Forward step (see lbm_kernels.cu), written in push form for one site x:
//   f*_i = (1 - w) f_i + w feq_i(rho, u),   w = 1/tau,
//   fluid link i: f_i(x + c_i, t+1) = f*_i;  wall link i: f_opp(i)(x, t+1) = f*_i;
//   iolet link i: f_opp(i)(x, t+1) = feq_opp(i)(rho_k(t), u).
// With lam(t) = dJ/df(t), the adjoint of the post-collision population is
//   lam*_i = lam_i(x + c_i, t+1) (fluid), lam_opp(i)(x, t+1) (wall), 0 (iolet),
// and the adjoint step is
//   lam_j(x, t) = (1 - w) lam*_j + w (a + b.(c_j - u)/rho) + g.(c_j - u)/rho
//                 + dj_t/df_j,
//   a = sum_i lam*_i feq_i/rho,  b = sum_i lam*_i dfeq_i/du,
//   dfeq_i/du = w_i rho (3 c_i + 9 (c_i.u) c_i - 3 u),
//   g = sum over iolet links of lam_opp(i)(x, t+1) dfeq_opp(i)(rho_k, u)/du.
// A velocity (Ladd) iolet link bounces like a wall less 6 w_i rho c_i.u_b:
//   lam*_i = lam_opp(i)(x, t+1), every lam_j gains -6 w_i (c_i.u_b) lam_opp(i),
//   dJ/dU_k(t) += -6 w_i rho weight(x) (c_i.n_k) lam_opp(i)(x, t+1).
// An interpolated (BFL) wall link p of x (the wall along c_opp(p) at the
// fraction q of the link, the fluid upstream site x_u = x + c_p):
//   f_p(x, t+1) = 2q f*_opp(p)(x) + (1 - 2q) f*_opp(p)(x_u)   (q < 1/2, x_u fluid),
//                 f*_opp(p)(x)                              (q < 1/2, no x_u),
//                 f*_opp(p)(x)/(2q) + (1 - 1/(2q)) f*_p(x)  (q >= 1/2),
// so lam*_opp(p)(x) = 2q, 1 or 1/(2q) times lam_p(x, t+1); for q >= 1/2
// lam*_p(x) gains (1 - 1/(2q)) lam_p(x, t+1); and for q < 1/2 the upstream
// site's lam*_opp(p)(x_u) = lam_opp(p)(x, t+1) gains (1 - 2q) lam_p(x, t+1),
// which x adds to the lam_opp(p) it stores, so that every site still reads
// one value per link (taken out again for dJ/df(t0)).
// Parameter derivatives of step t:
//   dJ/dtau      += sum_i lam*_i (f_i - feq_i) / tau^2,
//   dJ/drho_k(t) += sum over iolet-k links of lam_opp(i)(x, t+1) feq_opp(i)/rho_k,
// chained to mean, amp and phase of rho_k(t) = mean + amp sin(2 pi t/T + phase).
//
// In the pull form the adjoint state is kept in site form, lam[i][x]
// (float32), so the kernel is a pull like the forward step: lam*_i at x is
// read from the site that the forward table lists as the source of
// population opp(i) (the site x + c_i), or from x itself for wall and iolet
// links.  In the AA form (an AA context) the adjoint steps run in place on one
// buffer, alternating like the forward AA kernels (FORM_AA_EVEN / FORM_AA_ODD
// below).  Arithmetic is float32;
// the time accumulation of J and of every derivative is float64:
//   - J and dJ/dtau: the per-site terms (float) are summed over each thread
//     block in float, and the block totals go into one float64 pair per
//     block, added to by the same block at every step (a fixed grid, so the
//     summation order is fixed; GB300's FP64 pipe is narrow, so nothing per
//     site runs in float64);
//   - iolet derivatives: one float64 slot per (iolet site, direction) and
//     parameter, owned by one thread; reduced per iolet at the end.
// Nothing uses atomics, so gradients are bitwise reproducible.
#include <cuda_fp16.h>

#include <algorithm>

#include "lattice.h"
#include "lbm_internal.h"
#include "staging.cuh"

namespace hemelb_gb300 {
namespace {

constexpr int kBlock = 256;
// resident blocks per SM requested from the register allocator for the
// adjoint kernel without and with the wall-shear-stress objective term
#ifndef HGB_ADJ_MINB
#define HGB_ADJ_MINB 3
#endif
#ifndef HGB_ADJ_MINB_WSS
#define HGB_ADJ_MINB_WSS 2
#endif
// resident blocks per SM of the adjoint of an odd AA step
#ifndef HGB_ADJ_MINB_AA_ODD
#define HGB_ADJ_MINB_AA_ODD 3
#endif
// resident blocks per SM of the adjoint of an even AA step (bulk sites: no
// table, every access coalesced)
#ifndef HGB_ADJ_MINB_AA_EVEN
#define HGB_ADJ_MINB_AA_EVEN 4
#endif
// L2 prefetch distance, in blocks, of the bulk AA adjoint kernels (0: off):
// the even step's state and adjoint rows, the odd step's slot-table rows
// (and with HGB_ADJ_PF_ODD_ALL its state and adjoint rows too).  About one
// launch's resident blocks ahead (4 and 3 CTAs per SM).  Measured on the
// 10.8M-site tree (fp16 state, row order): 0.576 ms per adjoint step without,
// 0.556 even only, 0.571 odd table only, 0.554 both with the odd table only,
// 0.537 as built
#ifndef HGB_ADJ_PF_EVEN
#define HGB_ADJ_PF_EVEN 608
#endif
#ifndef HGB_ADJ_PF_ODD
#define HGB_ADJ_PF_ODD 456
#endif
#ifndef HGB_ADJ_PF_ODD_ALL
#define HGB_ADJ_PF_ODD_ALL 1
#endif
template <int HALF>
struct AdjLoad;
template <>
struct AdjLoad<0> {
    using T = float;
    static __device__ __forceinline__ float ld(const float *p, float) { return __ldg(p); }
};
// (the 16-bit forms scale by 2^-S with an explicit rounded product: a plain
// multiply may be fused with a later add in one adjoint kernel and not in
// another, and the AA and pull sweeps would then differ in the last bits)
template <>
struct AdjLoad<1> {
    using T = __half;
    static __device__ __forceinline__ float ld(const __half *p, float inv) {
        return __fmul_rn(__half2float(__ldg(p)), inv);
    }
};
template <>
struct AdjLoad<2> {
    using T = short;
    static __device__ __forceinline__ float ld(const short *p, float inv) {
        return __fmul_rn(__int_as_float(0x4B400000 + (int)__ldg(p)) - 12582912.0f, inv);
    }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block sum in a fixed order; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *part) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) part[w] = v;
    __syncthreads();
    v = threadIdx.x < kBlock / 32 ? part[threadIdx.x] : 0.0;
    if (w == 0) v = warp_sum(v);
    return v;
}

// float block sum of two per-thread values (the per-site terms of J and
// dJ/dtau), in a fixed order, valid in thread 0; the kernel converts the
// block totals to float64 for the accumulation over blocks and steps
__device__ __forceinline__ float2 block_sum_f2(float a, float b, float2 *part) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) part[w] = make_float2(a, b);
    __syncthreads();
    float2 v = threadIdx.x < kBlock / 32 ? part[threadIdx.x] : make_float2(0.f, 0.f);
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            v.x += __shfl_down_sync(0xffffffffu, v.x, o);
            v.y += __shfl_down_sync(0xffffffffu, v.y, o);
        }
    }
    return v;
}

template <int Q>
__device__ __forceinline__ float cdot(int i, float ux, float uy, float uz) {
    return cdir<Q>(i, 0) * ux + cdir<Q>(i, 1) * uy + cdir<Q>(i, 2) * uz;
}

// Wall-shear-stress objective term at site x (only launched for steps in
// the objective window): adds scale m d wss / d f_j to lam, returns m wss and
// adds the explicit tau derivative to *dtau.
// Non-equilibrium momentum flux sum_i (f_i - feq_i) c_i c_i (symmetric).
struct Stress {
    float xx, yy, zz, xy, xz, yz;
};

template <int Q>
__device__ __forceinline__ Stress stress(const float (&ne)[Q]) {
    Stress p{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int cx = cdir<Q>(i, 0), cy = cdir<Q>(i, 1), cz = cdir<Q>(i, 2);
        if (cx) p.xx += ne[i];
        if (cy) p.yy += ne[i];
        if (cz) p.zz += ne[i];
        if (cx * cy) p.xy += (cx * cy) * ne[i];
        if (cx * cz) p.xz += (cx * cz) * ne[i];
        if (cy * cz) p.yz += (cy * cz) * ne[i];
    }
    return p;
}

template <int Q, bool BFL>
__device__ __forceinline__ float wss_term(const DevLattice &L, const int (&s)[Q], const Stress &P,
                                          float rho, float ir, float ux, float uy, float uz,
                                          float usq15, float mx, float scale, float wss_dlog,
                                          float (&lam)[Q], float *dtau) {
    int wn0 = 0, wn1 = 0, wn2 = 0;
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (s[i] == -1 || (BFL && is_bfl(s[i]))) {  // half-way and interpolated walls
            wn0 += cdir<Q>(i, 0);
            wn1 += cdir<Q>(i, 1);
            wn2 += cdir<Q>(i, 2);
        }
    const float nn2 = (float)(wn0 * wn0 + wn1 * wn1 + wn2 * wn2);
    if (nn2 == 0.f) return 0.f;
    const float inn = 1.0f / sqrtf(nn2);
    const float n0 = wn0 * inn, n1 = wn1 * inn, n2 = wn2 * inn;
    const float coef = -(1.0f - 0.5f / L.tau);
    const float t0 = coef * (P.xx * n0 + P.xy * n1 + P.xz * n2);
    const float t1 = coef * (P.xy * n0 + P.yy * n1 + P.yz * n2);
    const float t2 = coef * (P.xz * n0 + P.yz * n1 + P.zz * n2);
    const float tn = t0 * n0 + t1 * n1 + t2 * n2;
    const float v0 = t0 - tn * n0, v1 = t1 - tn * n1, v2 = t2 - tn * n2;
    const float wss = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
    if (wss > 0.f) {
        *dtau += scale * mx * wss * wss_dlog;
        const float iv = 1.0f / wss;
        const float h0 = v0 * iv, h1 = v1 * iv, h2 = v2 * iv;
        float M[Q];
        float A = 0.f, Bx = 0.f, By = 0.f, Bz = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            M[i] = cdot<Q>(i, h0, h1, h2) * cdot<Q>(i, n0, n1, n2);
            const float cu = cdot<Q>(i, ux, uy, uz);
            const float wm = (float)wdir<Q>(i) * M[i];
            A += wm * (1.0f + 3.0f * cu + 4.5f * cu * cu - usq15);
            const float br = wm * rho;
            Bx += br * (3.0f * cdir<Q>(i, 0) + 9.0f * cu * cdir<Q>(i, 0) - 3.0f * ux);
            By += br * (3.0f * cdir<Q>(i, 1) + 9.0f * cu * cdir<Q>(i, 1) - 3.0f * uy);
            Bz += br * (3.0f * cdir<Q>(i, 2) + 9.0f * cu * cdir<Q>(i, 2) - 3.0f * uz);
        }
        const float sc = scale * mx * coef;
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float vx = (cdir<Q>(j, 0) - ux) * ir, vy = (cdir<Q>(j, 1) - uy) * ir,
                        vz = (cdir<Q>(j, 2) - uz) * ir;
            lam[j] += sc * (M[j] - (A + Bx * vx + By * vy + Bz * vz));
        }
    }
    return mx * wss;
}

// Storage forms of one adjoint step (the forward state P of time t and the
// adjoint buffers):
//   FORM_PULL     P in pull layout (gathered through the table); lam_next =
//                 lam(t+1) and lam_out = lam(t) in site form, two buffers.
//   FORM_AA_EVEN  the adjoint of an even (site-local) AA step: P in natural
//                 layout (own slots); one buffer, read as lam(t+1) in swapped
//                 form (every mu_i of site x in its own slot opp(i)) and
//                 written in place as lam(t) in site form; no table, except
//                 for iolet links and the wall-shear-stress normals.
//   FORM_AA_ODD   the adjoint of an odd AA step: P in swapped layout (its
//                 slots through the table); one buffer, read as lam(t+1) in
//                 site form (as FORM_PULL) and written in place as lam(t) in
//                 swapped form (lam_j(x) into slot opp(j) of the site x - c_j,
//                 or own slot j for a wall or iolet link): the slots read and
//                 written by a site are the same set, and no other site's.
// The adjoint of the AA form is AA-like itself (the streaming reversed), so
// the two alternate exactly as the forward kernels do; the arithmetic is the
// same in every form, so all give the same bits.
//   FORM_AA_SLOTS FORM_AA_ODD for the bulk sites (no iolet link), with tab(i)
//                 the slot-table entry of population i (DevLattice::slots,
//                 the AA odd-step slot): the state of population i is read
//                 at that slot, lam*_i at the slot of population opp(i) (the
//                 slot of population i of the site x + c_i in site form, or
//                 own slot opp(i) for a wall link), and lam_j is written at
//                 the slot of population j: no address arithmetic per site.
enum { FORM_PULL = 0, FORM_AA_EVEN = 1, FORM_AA_ODD = 2, FORM_AA_SLOTS = 3 };

// The adjoint of step t at one site x (lam(t) at x from lam(t+1) and the
// state P of time t); tab(i) is the table entry of population i at x (from
// registers or global memory).  Adds the
// site's terms of J and dJ/dtau to j_site and dtau_site (float).
template <int Q, int HALF, bool WSS, bool IO, int FORM, bool BFL, typename Tab, typename TabOut>
__device__ __forceinline__ void adjoint_site(const DevLattice &L, const typename AdjLoad<HALF>::T *__restrict__ P,
                                             const float *lam_next, float *lam_out, const AdjStep &st,
                                             const AdjObjective &obj, int x, const Tab &tab,
                                             const TabOut &tab_out, double *__restrict__ io_acc, float &j_site,
                                             float &dtau_site) {
    using R = AdjLoad<HALF>;
    const unsigned np = (unsigned)L.npad;
    float ne[Q];
    ne[0] = R::ld(P + x, L.inv_scale);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        unsigned e;
        if (FORM == FORM_AA_EVEN) {
            e = (unsigned)i * np + (unsigned)x;
        } else if (FORM == FORM_AA_SLOTS) {
            e = (unsigned)tab(i);
        } else {
            const int si = tab(i);
            const unsigned a = FORM == FORM_PULL ? (unsigned)i : (unsigned)opp(i);
            const unsigned b = FORM == FORM_PULL ? (unsigned)opp(i) : (unsigned)i;
            e = si >= 0 ? a * np + (unsigned)si : b * np + (unsigned)x;
        }
        ne[i] = R::ld(P + e, L.inv_scale);
    }
    if (BFL) {
        // interpolated walls: the slot of a q < 1/2 link p with a fluid
        // upstream site holds 2q f*; f_p(t) adds (1 - 2q) times the
        // population opp(p) pulled from that site (the forward gather)
#pragma unroll
        for (int p = 1; p < Q; ++p) {
            const int sp = tab(p);
            if (is_bfl(sp)) {
                const float qv = bfl_q(sp);
                if (qv < 0.5f && tab(opp(p)) >= 0) ne[p] = fmaf(1.0f - 2.0f * qv, ne[opp(p)], ne[p]);
            }
        }
    }
    float drho = ne[0], jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float sum = ne[i] + ne[i + 1], dif = ne[i] - ne[i + 1];
        drho += sum;
        if (cdir<Q>(i, 0)) jx += cdir<Q>(i, 0) * dif;
        if (cdir<Q>(i, 1)) jy += cdir<Q>(i, 1) * dif;
        if (cdir<Q>(i, 2)) jz += cdir<Q>(i, 2) * dif;
    }
    const float rho = L.rho0 + drho;
    const float ir = 1.0f / rho;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
    // non-equilibrium parts f_i - feq_i (in place of the deviations)
    ne[0] -= (float)wdir<Q>(0) * (drho - rho * usq15);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = (float)wdir<Q>(i);
        const float cu = cdot<Q>(i, ux, uy, uz);
        const float sym = w * (drho + rho * fmaf(4.5f * cu, cu, -usq15));
        const float asym = 3.0f * w * rho * cu;
        ne[i] -= sym + asym;
        ne[i + 1] -= sym - asym;
    }
    Stress Pst{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (WSS) Pst = stress<Q>(ne);
    // (no ordering fence here: overlapping the forward-state and adjoint
    // gathers is worth more than the registers it costs; fencing them
    // apart measured 1.50 ms per step against 1.06 ms)
    // adjoint of the post-collision populations, with the iolet terms
    // (all gathers issued first, then the pairwise sums: keeping the loads
    // back to back measured faster than accumulating as they arrive)
    float ls[Q];
    float gx = 0.f, gy = 0.f, gz = 0.f, gvel = 0.f;
    const bool has_next = lam_next != nullptr;
    ls[0] = has_next ? lam_next[x] : 0.f;
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        ls[i] = 0.f;
        if (FORM == FORM_AA_EVEN && !IO) {
            // (no iolet link: mu_i in the own slot opp(i) for every link)
            if (has_next) ls[i] = lam_next[(unsigned)opp(i) * np + (unsigned)x];
            continue;
        }
        if (FORM == FORM_AA_SLOTS) {
            // (no iolet link: lam*_i at the slot of population opp(i))
            if (has_next) ls[i] = lam_next[(unsigned)tab(opp(i))];
            continue;
        }
        const int sp = tab(opp(i));  // link i of x: >= 0 -> the site x + c_i
        if (has_next) {
            if (sp >= 0) {
                ls[i] = FORM == FORM_AA_EVEN ? lam_next[(unsigned)opp(i) * np + (unsigned)x]
                                             : lam_next[(unsigned)i * np + (unsigned)sp];
            } else if (BFL && is_bfl(sp)) {
                // interpolated wall along c_i (population p = opp(i) arrives
                // from the wall side): f*_i feeds f_p(x, t+1) with 2q (q < 1/2
                // and a fluid upstream site), 1 (q < 1/2, none) or 1/(2q)
                // (a rounded product: left to the code generator, the multiply
                // may fuse with a later add in one kernel and not in another,
                // and the AA and pull sweeps would no longer agree to the bit)
                const float qv = bfl_q(sp);
                const float lo = lam_next[(unsigned)opp(i) * np + (unsigned)x];
                ls[i] = __fmul_rn(qv < 0.5f ? (tab(i) >= 0 ? 2.0f * qv : 1.0f) : 0.5f / qv, lo);
            } else if (!IO || sp == -1) {
                ls[i] = lam_next[(unsigned)opp(i) * np + (unsigned)x];
            } else if ((st.io.vel_mask >> (-2 - sp)) & 1ull) {
                // velocity iolet: the link bounces f*_i like a wall, less
                // Ladd's moving-boundary term 6 w_i rho c_i.u_b, u_b = weight(x)
                // U_k(t) n_k, which feeds back through rho into every lam_j
                // (d rho / d f_j = 1) and into dJ/dU_k(t)
                const float lo = lam_next[(unsigned)opp(i) * np + (unsigned)x];
                const int k = -2 - sp;
                ls[i] = lo;
                const float cn = cdot<Q>(i, st.io.nrm[k][0], st.io.nrm[k][1], st.io.nrm[k][2]);
                const float wl = 6.0f * (float)wdir<Q>(i) * L.vel_weight[x - L.n_bulk] * cn * lo;
                gvel -= wl * st.io.rho[k];
                const float du = -wl * rho;
                const size_t slot = (size_t)(x - L.n_bulk) * (Q - 1) + (i - 1);
                const size_t plane = (size_t)(L.n - L.n_bulk) * (Q - 1);
                io_acc[slot] += (double)du;
                io_acc[plane + slot] += (double)du * st.dsin[k];
                io_acc[2 * plane + slot] += (double)du * st.dacos[k];
            } else {
                const float lo = lam_next[(unsigned)opp(i) * np + (unsigned)x];
                const int k = -2 - sp;
                const int o = opp(i);
                const float rk = st.io.rho[k];
                const float cu = cdot<Q>(o, ux, uy, uz);
                const float wo = (float)wdir<Q>(o);
                const float drk = lo * wo * (1.0f + 3.0f * cu + 4.5f * cu * cu - usq15);
                const float gc = lo * wo * rk;
                gx += gc * (3.0f * cdir<Q>(o, 0) + 9.0f * cu * cdir<Q>(o, 0) - 3.0f * ux);
                gy += gc * (3.0f * cdir<Q>(o, 1) + 9.0f * cu * cdir<Q>(o, 1) - 3.0f * uy);
                gz += gc * (3.0f * cdir<Q>(o, 2) + 9.0f * cu * cdir<Q>(o, 2) - 3.0f * uz);
                const size_t slot = (size_t)(x - L.n_bulk) * (Q - 1) + (i - 1);
                const size_t plane = (size_t)(L.n - L.n_bulk) * (Q - 1);
                io_acc[slot] += (double)drk;
                io_acc[plane + slot] += (double)drk * st.dsin[k];
                io_acc[2 * plane + slot] += (double)drk * st.dacos[k];
            }
        }
    }
    if (BFL && has_next) {
        // q >= 1/2: f*_p feeds f_p(x, t+1) as well, with 1 - 1/(2q)
#pragma unroll
        for (int p = 1; p < Q; ++p) {
            const int sp = tab(p);
            if (is_bfl(sp)) {
                const float qv = bfl_q(sp);
                if (qv >= 0.5f)
                    ls[p] = fmaf(1.0f - 0.5f / qv, lam_next[(unsigned)p * np + (unsigned)x], ls[p]);
            }
        }
    }
    // a = sum_i lam*_i feq_i/rho, b = sum_i lam*_i dfeq_i/du (pairwise),
    // dt = sum_i lam*_i (f_i - feq_i)
    float a = (float)wdir<Q>(0) * ls[0] * (1.0f - usq15);
    float bx = 0.f, by = 0.f, bz = 0.f;
    float sb = (float)wdir<Q>(0) * ls[0];
    float dt = ls[0] * ne[0];
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float w = (float)wdir<Q>(i);
        const float cu = cdot<Q>(i, ux, uy, uz);
        const float sum = ls[i] + ls[i + 1], dif = ls[i] - ls[i + 1];
        a += w * fmaf(sum, 1.0f + fmaf(4.5f * cu, cu, -usq15), 3.0f * cu * dif);
        const float bc = w * fmaf(9.0f * cu, sum, 3.0f * dif);
        if (cdir<Q>(i, 0)) bx += cdir<Q>(i, 0) * bc;
        if (cdir<Q>(i, 1)) by += cdir<Q>(i, 1) * bc;
        if (cdir<Q>(i, 2)) bz += cdir<Q>(i, 2) * bc;
        sb += w * sum;
        dt = fmaf(ls[i], ne[i], dt);
        dt = fmaf(ls[i + 1], ne[i + 1], dt);
    }
    // b = rho (bc-sum - 3 u sb)
    bx = rho * (bx - 3.0f * ux * sb);
    by = rho * (by - 3.0f * uy * sb);
    bz = rho * (bz - 3.0f * uz * sb);
    dtau_site = dt * obj.inv_tau2_f;
    const float om = L.omega, omc = 1.0f - L.omega;
    // lam_j = omc lam*_j + om a + Bv.(c_j - u), Bv = (om b + g)/rho
    const float Bx = (om * bx + gx) * ir, By = (om * by + gy) * ir, Bz = (om * bz + gz) * ir;
    const float base = om * a - (Bx * ux + By * uy + Bz * uz) + gvel;
    float lam[Q];
    lam[0] = fmaf(omc, ls[0], base);
#pragma unroll
    for (int i = 1; i < Q; i += 2) {
        const float bcj = cdot<Q>(i, Bx, By, Bz);
        lam[i] = fmaf(omc, ls[i], base + bcj);
        lam[i + 1] = fmaf(omc, ls[i + 1], base - bcj);
    }
    // explicit objective terms of the state f(t)
    if (obj.active) {
        // a non-zero weight, tested on its bits (no float64 instruction)
        const double mxd = obj.weight[x];
        if ((__double_as_longlong(mxd) << 1) != 0) {
            const float mx = (float)mxd;
            if (WSS) {
                int s[Q];
                s[0] = 0;
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    if (FORM == FORM_AA_SLOTS)  // a wall link reads the own slot i
                        s[i] = (unsigned)tab(i) == (unsigned)i * np + (unsigned)x ? -1 : 0;
                    else
                        s[i] = tab(i);
                }
                j_site = wss_term<Q, BFL>(L, s, Pst, rho, ir, ux, uy, uz, usq15, mx, obj.scale_f,
                                     obj.wss_dlog_f, lam, &dtau_site);
            } else if (obj.kind == 1) {
                // m (rho - rho0): the host adds rho0 sum(m) per state in
                // float64, so the float block sums carry only the small part
                j_site = mx * drho;
                const float sm = obj.scale_f * mx;
#pragma unroll
                for (int j = 0; j < Q; ++j) lam[j] += sm;
            }
        }
    }
    if (BFL) {
        // lam_opp(p)(x, t) is read by the upstream site x + c_p (fluid, q <
        // 1/2) as its lam* of population opp(p), whose post-collision value
        // also fed f_p(x, t) with (1 - 2q): it is stored with that term added
        // (k_lam_to_caller takes it out again for dJ/df(t0))
#pragma unroll
        for (int p = 1; p < Q; ++p) {
            const int sp = tab(p);
            if (is_bfl(sp)) {
                const float qv = bfl_q(sp);
                if (qv < 0.5f && tab(opp(p)) >= 0) lam[opp(p)] = fmaf(1.0f - 2.0f * qv, lam[p], lam[opp(p)]);
            }
        }
    }
    if (FORM == FORM_AA_ODD) {
        __stcs(lam_out + x, lam[0]);
#pragma unroll
        for (int j = 1; j < Q; ++j) {
            const int sj = tab_out(j);
            __stcs(lam_out + (sj >= 0 ? (unsigned)opp(j) * np + (unsigned)sj : (unsigned)j * np + (unsigned)x),
                   lam[j]);
        }
    } else if (FORM == FORM_AA_SLOTS) {
        __stcs(lam_out + x, lam[0]);
#pragma unroll
        for (int j = 1; j < Q; ++j) __stcs(lam_out + (unsigned)tab_out(j), lam[j]);
    } else {
#pragma unroll
        for (int j = 0; j < Q; ++j) __stcs(lam_out + (unsigned)j * np + (unsigned)x, lam[j]);
    }
}

// One adjoint step over the sites [x_begin, x_end): the bulk sites (no
// iolet link, IO = false) or the iolet sites (IO = true), one block per
// 256-site tile.  WSS = the wall-shear-stress objective term is active at
// this step.
template <int Q, int HALF, bool WSS, bool IO, bool BFL = false>
__global__ void __launch_bounds__(kBlock, WSS ? HGB_ADJ_MINB_WSS : HGB_ADJ_MINB)
k_adjoint(const DevLattice L, const typename AdjLoad<HALF>::T *__restrict__ P,
          const float *__restrict__ lam_next, float *__restrict__ lam_out, const AdjStep st,
          const AdjObjective obj, int x_begin, int x_end, double *__restrict__ acc_block,
          double *__restrict__ io_acc) {
    __shared__ float2 part[kBlock / 32];
    const int x = x_begin + blockIdx.x * kBlock + threadIdx.x;
    const unsigned np = (unsigned)L.npad;
    float j_site = 0.f, dtau_site = 0.f;
    if (x < x_end) {
        int s[Q];
        s[0] = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) s[i] = __ldg(L.tab + (unsigned)(i - 1) * np + (unsigned)x);
        auto tab = [&](int i) { return s[i]; };
        adjoint_site<Q, HALF, WSS, IO, FORM_PULL, BFL>(L, P, lam_next, lam_out, st, obj, x, tab, tab, io_acc,
                                                       j_site, dtau_site);
    }
    const float2 bsum = block_sum_f2(j_site, dtau_site, part);
    if (threadIdx.x == 0) {
        const int b = (x_begin == 0 ? 0 : (L.n_bulk + kBlock - 1) / kBlock) + blockIdx.x;
        acc_block[2 * b] += (double)bsum.x;
        acc_block[2 * b + 1] += (double)bsum.y;
    }
}

// One adjoint step of the AA form (FORM_AA_EVEN or FORM_AA_ODD, see above) over
// the sites [x_begin, x_end), in place on the one adjoint buffer lam (read as
// lam(t+1), written as lam(t)); tiles and block sums as in k_adjoint.
template <int Q, int HALF, bool WSS, bool IO, bool ODD, bool BFL = false>
__global__ void __launch_bounds__(kBlock, WSS ? HGB_ADJ_MINB_WSS
                                              : IO ? HGB_ADJ_MINB : ODD ? HGB_ADJ_MINB_AA_ODD : HGB_ADJ_MINB_AA_EVEN)
k_adjoint_aa(const DevLattice L, const typename AdjLoad<HALF>::T *__restrict__ P, float *lam, int has_next,
             const AdjStep st, const AdjObjective obj, int x_begin, int x_end, double *__restrict__ acc_block,
             double *__restrict__ io_acc) {
    __shared__ float2 part[kBlock / 32];
    const int x = x_begin + blockIdx.x * kBlock + threadIdx.x;
    const unsigned np = (unsigned)L.npad;
    float j_site = 0.f, dtau_site = 0.f;
    if (!IO && (ODD ? HGB_ADJ_PF_ODD : HGB_ADJ_PF_EVEN) > 0) {
        const unsigned x0 =
            (unsigned)x_begin + (blockIdx.x + (ODD ? HGB_ADJ_PF_ODD : HGB_ADJ_PF_EVEN)) * (unsigned)kBlock;
        const int r = (int)threadIdx.x;
        if (ODD) {
            prefetch_rows(L.slots, 4u, np, Q - 1, x0, (unsigned)x_end, np, r);
            if (HGB_ADJ_PF_ODD_ALL) {
                prefetch_rows(P, sizeof(typename AdjLoad<HALF>::T), np, Q, x0, (unsigned)x_end, np, r - (Q - 1));
                prefetch_rows(lam, 4u, np, Q, x0, (unsigned)x_end, np, r - (2 * Q - 1));
            }
        } else {
            prefetch_rows(P, sizeof(typename AdjLoad<HALF>::T), np, Q, x0, (unsigned)x_end, np, r);
            prefetch_rows(lam, 4u, np, Q, x0, (unsigned)x_end, np, r - Q);
        }
    }
    if (x < x_end) {
        const float *lin = has_next ? lam : nullptr;
        // the table entries again for the swapped-form stores of an odd step:
        // a volatile load is not merged with the first one, so the entries
        // need not stay in registers through the whole site
        auto reload = [&](int i) {
            int v;
            asm volatile("ld.global.nc.s32 %0, [%1];" : "=r"(v) : "l"(L.tab + (unsigned)(i - 1) * np + (unsigned)x));
            return v;
        };
        if (ODD && !IO) {
            // bulk sites of an odd step: every access through the slot table
            unsigned e[Q];
            e[0] = (unsigned)x;
#pragma unroll
            for (int i = 1; i < Q; ++i) e[i] = __ldg(L.slots + (unsigned)(i - 1) * np + (unsigned)x);
            auto tab = [&](int i) { return (int)e[i]; };
            auto reload_slot = [&](int i) {
                unsigned v;
                asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(L.slots + (unsigned)(i - 1) * np + (unsigned)x));
                return (int)v;
            };
            adjoint_site<Q, HALF, WSS, false, FORM_AA_SLOTS, false>(L, P, lin, lam, st, obj, x, tab, reload_slot,
                                                                    io_acc, j_site, dtau_site);
        } else if (ODD || IO) {
            int s[Q];
            s[0] = 0;
#pragma unroll
            for (int i = 1; i < Q; ++i) s[i] = __ldg(L.tab + (unsigned)(i - 1) * np + (unsigned)x);
            auto tab = [&](int i) { return s[i]; };
            adjoint_site<Q, HALF, WSS, IO, ODD ? FORM_AA_ODD : FORM_AA_EVEN, BFL>(L, P, lin, lam, st, obj, x, tab,
                                                                                 reload, io_acc, j_site,
                                                                                 dtau_site);
        } else {
            // even step of a bulk site: the table only for the wall normals
            // of the wall-shear-stress term
            auto tab = [&](int i) { return __ldg(L.tab + (unsigned)(i - 1) * np + (unsigned)x); };
            adjoint_site<Q, HALF, WSS, false, FORM_AA_EVEN, false>(L, P, lin, lam, st, obj, x, tab, tab, io_acc,
                                                                  j_site, dtau_site);
        }
    }
    const float2 bsum = block_sum_f2(j_site, dtau_site, part);
    if (threadIdx.x == 0) {
        const int b = (x_begin == 0 ? 0 : (L.n_bulk + kBlock - 1) / kBlock) + blockIdx.x;
        acc_block[2 * b] += (double)bsum.x;
        acc_block[2 * b + 1] += (double)bsum.y;
    }
}

// J and dJ/dtau: sum of the per-block accumulators in a fixed order
__global__ void __launch_bounds__(kBlock)
k_acc_final(const double *__restrict__ acc_block, int nblocks, double *__restrict__ out) {
    __shared__ double part[kBlock / 32];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += kBlock) {
        a += acc_block[2 * i];
        b += acc_block[2 * i + 1];
    }
    a = block_sum(a, part);
    b = block_sum(b, part);
    if (threadIdx.x == 0) {
        out[0] = a;
        out[1] = b;
    }
}

// per-iolet derivatives: block k sums, over the iolet sites and the
// directions whose link is iolet k, the three accumulated parameters
template <int Q>
__global__ void __launch_bounds__(kBlock)
k_io_final(const DevLattice L, const double *__restrict__ io_acc, double *__restrict__ out) {
    __shared__ double part[kBlock / 32];
    const int k = blockIdx.x;
    const int nio = L.n - L.n_bulk;
    const size_t plane = (size_t)nio * (Q - 1);
    const unsigned np = (unsigned)L.npad;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (size_t e = threadIdx.x; e < plane; e += kBlock) {
        const int xi = (int)(e / (Q - 1));
        const int i = (int)(e % (Q - 1)) + 1;
        const int x = L.n_bulk + xi;
        // link i of x is iolet k when the table entry of population opp(i) is -2 - k
        if (L.tab[(unsigned)(opp(i) - 1) * np + (unsigned)x] == -2 - k) {
            s0 += io_acc[e];
            s1 += io_acc[plane + e];
            s2 += io_acc[2 * plane + e];
        }
    }
    s0 = block_sum(s0, part);
    s1 = block_sum(s1, part);
    s2 = block_sum(s2, part);
    if (threadIdx.x == 0) {
        out[k] = s0;
        out[L.n_iolets + k] = s1;
        out[2 * L.n_iolets + k] = s2;
    }
}

template <int Q>
__global__ void __launch_bounds__(kBlock)
k_lam_to_caller(const DevLattice L, const float *__restrict__ lam, double *__restrict__ out) {
    const int x = blockIdx.x * kBlock + threadIdx.x;
    if (x >= L.n) return;
    const int64_t xc = L.perm[x];
    float v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) v[i] = lam[(int64_t)i * L.npad + x];
    if (L.bfl && x >= L.n_bulk) {
        // the stored lam_opp(p) of a q < 1/2 interpolated link with a fluid
        // upstream site carries (1 - 2q) lam_p for that site: take it out
        int s[Q];
        s[0] = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) s[i] = L.tab[(int64_t)(i - 1) * L.npad + x];
#pragma unroll
        for (int p = 1; p < Q; ++p)
            if (is_bfl(s[p])) {
                const float qv = bfl_q(s[p]);
                if (qv < 0.5f && s[opp(p)] >= 0) v[opp(p)] = fmaf(-(1.0f - 2.0f * qv), v[p], v[opp(p)]);
            }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(int64_t)i * L.n + xc] = (double)v[i];
}

template <int Q, int HALF, bool WSS>
cudaError_t adjoint_impl(const DevLattice &L, const void *P, const float *lam_next, float *lam_out,
                         const AdjStep &st, const AdjObjective &obj, double *acc_block,
                         double *io_acc, cudaStream_t s, cudaStream_t t) {
    using T = typename AdjLoad<HALF>::T;
    const int nb = L.n_bulk, ni = L.n - L.n_bulk;
    if (nb > 0)
        k_adjoint<Q, HALF, WSS, false><<<(nb + kBlock - 1) / kBlock, kBlock, 0, s>>>(
            L, (const T *)P, lam_next, lam_out, st, obj, 0, nb, acc_block, io_acc);
    if (ni > 0 && L.bfl)
        k_adjoint<Q, HALF, WSS, true, true><<<(ni + kBlock - 1) / kBlock, kBlock, 0, t>>>(
            L, (const T *)P, lam_next, lam_out, st, obj, nb, L.n, acc_block, io_acc);
    else if (ni > 0)
        k_adjoint<Q, HALF, WSS, true><<<(ni + kBlock - 1) / kBlock, kBlock, 0, t>>>(
            L, (const T *)P, lam_next, lam_out, st, obj, nb, L.n, acc_block, io_acc);
    return cudaGetLastError();
}

template <int Q, int HALF>
cudaError_t adjoint_q(const DevLattice &L, const void *P, const float *lam_next, float *lam_out,
                      const AdjStep &st, const AdjObjective &obj, double *acc_block, double *io_acc,
                      cudaStream_t s, cudaStream_t t) {
    if (obj.active && obj.kind == 0)
        return adjoint_impl<Q, HALF, true>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t);
    return adjoint_impl<Q, HALF, false>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t);
}

template <int Q, int HALF, bool WSS, bool ODD>
cudaError_t adjoint_aa_impl(const DevLattice &L, const void *P, float *lam, bool has_next, const AdjStep &st,
                            const AdjObjective &obj, double *acc_block, double *io_acc, cudaStream_t s,
                            cudaStream_t t) {
    using T = typename AdjLoad<HALF>::T;
    const int nb = L.n_bulk, ni = L.n - L.n_bulk;
    if (nb > 0)
        k_adjoint_aa<Q, HALF, WSS, false, ODD><<<(nb + kBlock - 1) / kBlock, kBlock, 0, s>>>(
            L, (const T *)P, lam, has_next ? 1 : 0, st, obj, 0, nb, acc_block, io_acc);
    if (ni > 0 && L.bfl)
        k_adjoint_aa<Q, HALF, WSS, true, ODD, true><<<(ni + kBlock - 1) / kBlock, kBlock, 0, t>>>(
            L, (const T *)P, lam, has_next ? 1 : 0, st, obj, nb, L.n, acc_block, io_acc);
    else if (ni > 0)
        k_adjoint_aa<Q, HALF, WSS, true, ODD><<<(ni + kBlock - 1) / kBlock, kBlock, 0, t>>>(
            L, (const T *)P, lam, has_next ? 1 : 0, st, obj, nb, L.n, acc_block, io_acc);
    return cudaGetLastError();
}

template <int Q, int HALF>
cudaError_t adjoint_aa_q(const DevLattice &L, const void *P, bool p_swapped, float *lam, bool has_next,
                         const AdjStep &st, const AdjObjective &obj, double *acc_block, double *io_acc,
                         cudaStream_t s, cudaStream_t t) {
    const bool wss = obj.active && obj.kind == 0;
    if (p_swapped)
        return wss ? adjoint_aa_impl<Q, HALF, true, true>(L, P, lam, has_next, st, obj, acc_block, io_acc, s, t)
                   : adjoint_aa_impl<Q, HALF, false, true>(L, P, lam, has_next, st, obj, acc_block, io_acc, s, t);
    return wss ? adjoint_aa_impl<Q, HALF, true, false>(L, P, lam, has_next, st, obj, acc_block, io_acc, s, t)
               : adjoint_aa_impl<Q, HALF, false, false>(L, P, lam, has_next, st, obj, acc_block, io_acc, s, t);
}

}  // namespace

cudaError_t launch_adjoint_aa(const DevLattice &L, const void *P, bool p_swapped, float *lam, bool has_next,
                              const AdjStep &st, const AdjObjective &obj, double *acc_block, double *io_acc,
                              cudaStream_t s, cudaStream_t t) {
    if (L.n == 0) return cudaSuccess;
    if (L.q == 15)
        return L.storage == 2 ? adjoint_aa_q<15, 2>(L, P, p_swapped, lam, has_next, st, obj, acc_block, io_acc, s, t)
             : L.storage      ? adjoint_aa_q<15, 1>(L, P, p_swapped, lam, has_next, st, obj, acc_block, io_acc, s, t)
                              : adjoint_aa_q<15, 0>(L, P, p_swapped, lam, has_next, st, obj, acc_block, io_acc, s, t);
    return L.storage == 2 ? adjoint_aa_q<19, 2>(L, P, p_swapped, lam, has_next, st, obj, acc_block, io_acc, s, t)
         : L.storage      ? adjoint_aa_q<19, 1>(L, P, p_swapped, lam, has_next, st, obj, acc_block, io_acc, s, t)
                          : adjoint_aa_q<19, 0>(L, P, p_swapped, lam, has_next, st, obj, acc_block, io_acc, s, t);
}

// blocks of the bulk launch plus blocks of the iolet-site launch
int adjoint_blocks(const DevLattice &L) {
    return (L.n_bulk + kBlock - 1) / kBlock + (L.n - L.n_bulk + kBlock - 1) / kBlock;
}

cudaError_t launch_adjoint(const DevLattice &L, const void *P, const float *lam_next, float *lam_out,
                           const AdjStep &st, const AdjObjective &obj, double *acc_block,
                           double *io_acc, cudaStream_t s, cudaStream_t t) {
    if (L.n == 0) return cudaSuccess;
    if (L.q == 15)
        return L.storage == 2 ? adjoint_q<15, 2>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t)
             : L.storage      ? adjoint_q<15, 1>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t)
                              : adjoint_q<15, 0>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t);
    return L.storage == 2 ? adjoint_q<19, 2>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t)
         : L.storage      ? adjoint_q<19, 1>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t)
                          : adjoint_q<19, 0>(L, P, lam_next, lam_out, st, obj, acc_block, io_acc, s, t);
}

cudaError_t launch_adjoint_final(const DevLattice &L, const double *acc_block, const double *io_acc,
                                 double *out, cudaStream_t s) {
    k_acc_final<<<1, kBlock, 0, s>>>(acc_block, adjoint_blocks(L), out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || L.n_iolets == 0) return e;
    if (L.q == 15)
        k_io_final<15><<<L.n_iolets, kBlock, 0, s>>>(L, io_acc, out + 2);
    else
        k_io_final<19><<<L.n_iolets, kBlock, 0, s>>>(L, io_acc, out + 2);
    return cudaGetLastError();
}

cudaError_t launch_lam_to_caller(const DevLattice &L, const float *lam, double *out, cudaStream_t s) {
    if (L.n == 0) return cudaSuccess;
    const unsigned g = (unsigned)((L.n + kBlock - 1) / kBlock);
    if (L.q == 15)
        k_lam_to_caller<15><<<g, kBlock, 0, s>>>(L, lam, out);
    else
        k_lam_to_caller<19><<<g, kBlock, 0, s>>>(L, lam, out);
    return cudaGetLastError();
}

}  // namespace hemelb_gb300
