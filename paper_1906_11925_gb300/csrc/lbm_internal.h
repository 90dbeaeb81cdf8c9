// Internal interface between the host side of libhemelb_gb300 (lbm_host.cpp)
// and its CUDA kernels (lbm_kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace hemelb_gb300 {

constexpr int kMaxIolets = 64;

// Sites per tile of the table-staged pull kernel (one site per thread).
constexpr int kTile = 256;

// Interpolated (BFL) wall links in the pull table: the entry of population
// p whose link opp(p) is a wall at fluid fraction q != 1/2 is
// INT32_MIN + round(q 2^24) (q in (0, 1], a multiple of 2^-24).  Such sites
// come after the bulk sites ([n_bulk, n)).  The slot the step reads back for
// p (own slot opp(p)) holds, for q < 1/2 with a fluid upstream site, 2q f*
// (the other part, (1 - 2q) times the population opp(p) pulled from the
// upstream site, is added when the site gathers); otherwise the whole
// interpolated value.
#if defined(__CUDACC__)
#define HGB_BFL_HD __host__ __device__
#else
#define HGB_BFL_HD
#endif
constexpr int32_t kBflMax = (int32_t)(0x80000000u + (1u << 24));
HGB_BFL_HD inline bool is_bfl(int32_t e) { return e <= kBflMax; }
HGB_BFL_HD inline float bfl_q(int32_t e) { return (float)((uint32_t)e ^ 0x80000000u) * (1.0f / 16777216.0f); }
HGB_BFL_HD inline int32_t bfl_code(double q) {
    const double k = q * 16777216.0 + 0.5;
    uint32_t u = (uint32_t)(k < 1.0 ? 1.0 : (k > 16777216.0 ? 16777216.0 : k));
    return (int32_t)(0x80000000u + u);
}

// Where population i of site x is stored (see src_slot in lbm_kernels.cu).
enum Layout { LAYOUT_PULL = 0, LAYOUT_NATURAL = 1, LAYOUT_AA_SWAPPED = 2 };

// Iolet densities of one step, evaluated on the host in float64 and passed
// by value: drho[k] = rho_k(t) - rho0 (rounded once to float, so that the
// small pressure differences keep their relative precision), rho[k] = rho_k(t).
// For a velocity iolet (bit k of vel_mask) rho[k] carries the speed U_k(t)
// instead, and nrm[k] its unit inward normal.
struct IoletStep {
    float drho[kMaxIolets];
    float rho[kMaxIolets];
    float nrm[kMaxIolets][3];
    unsigned long long vel_mask;
};

// Device-side description of one simulation, passed by value to launchers.
//
// Kernel table layout (internal order: Morton order of the sites without
// iolet links, then Morton order of those with one; planes of length npad):
//   tab[(i - 1) * npad + x], i = 1..q-1, is the pull source of population i
//   at site x: >= 0 -> population i of site tab (the site x - c_i);
//   -1 -> wall link opp(i) at x (read own slot opp(i), halfway bounce-back);
//   -2 - k -> iolet-k link opp(i) at x (read own slot opp(i), which the
//   previous step filled with the iolet equilibrium).
// Populations: f[i * npad + x] as float (fp32 storage), __half bits (fp16
// storage) or int16 (fixed point) holding the deviation from w_i rho0 (times
// 2^S for the 16-bit forms).
struct DevLattice {
    int q;
    int storage;     // 0 fp32, 1 fp16, 2 int16
    int n;           // sites
    int n_bulk;      // sites [0, n_bulk) have no iolet link; [n_bulk, n) have
    int64_t npad;    // plane length (multiple of 128)
    float omega;     // 1 / tau
    float tau;
    float rho0;
    float scale;     // 2^S (fp16 store multiplier)
    float inv_scale; // 2^-S
    int n_iolets;
    const int32_t *tab;           // [q-1][npad]
    const int32_t *perm;          // [n] internal -> caller index
    int *err;                     // device flag: a bounded wait in a kernel timed out
    // Slot table of the bulk sites [0, n_bulk), [q-1][npad]: slots[(i - 1) *
    // npad + x] is the element offset in the population buffer that the bulk
    // step kernel reads population i of site x from: pull streaming, the
    // slot i * npad + tab of the pull source (opp(i) * npad + x for a wall
    // link); AA streaming, the slot that the odd step reads and writes back,
    // opp(i) * npad + tab (i * npad + x for a wall link).  The same
    // information as tab, with the address arithmetic done once at create.
    const uint32_t *slots;
    const float *vel_weight;      // [n - n_bulk] velocity-iolet weight of the iolet sites
    int bfl;                      // the table holds interpolated wall links
};

// Slots after the last plane of a population buffer that hold guard words
// (the plane padding [n, npad) holds them too).
constexpr int64_t kGuardSlots = 128;

// Instability check of the stored state f (any layout): on a non-finite
// slot, rho <= 0 or |u| > u_max at a site, stores tag in *flag if *flag is 0.
cudaError_t launch_stability(const DevLattice &L, const void *f, float u_max, int tag, int *flag,
                             cudaStream_t s);

// Write (check = false) or compare (check = true; mismatch: *flag = 1) the
// guard words of the population buffer f.
cudaError_t launch_guards(const DevLattice &L, void *f, bool check, int *flag, cudaStream_t s);

// One fused pull collide-and-stream step from fin into fout.  The iolet
// densities come from io, or, when rho_io (device, float64 [n_iolets]) is not
// null, from rho_io.
// A second stream on which the small launch of the sites after the bulk runs
// alongside the bulk launch (the two touch disjoint slots): fork records on
// the main stream and the side stream waits for it, join records on the side
// stream and the main stream waits for it.  Null: both launches in order on
// the main stream.
struct SideStream {
    cudaStream_t s;
    cudaEvent_t fork, join;
};

// io_dev (device, one IoletStep), when not null, replaces io: the steps of a
// CUDA graph read their iolet values from memory the host refills per replay.
cudaError_t launch_step(const DevLattice &L, const void *fin, void *fout, const IoletStep &io,
                        const double *rho_io, cudaStream_t s, const SideStream *side = nullptr,
                        const IoletStep *io_dev = nullptr);

// One in-place AA-pattern step on the single buffer A: the even kernel
// (A in natural layout -> swapped) or the odd kernel (swapped -> natural).
cudaError_t launch_step_aa(const DevLattice &L, void *A, bool odd, const IoletStep &io,
                           const double *rho_io, cudaStream_t s, const SideStream *side = nullptr,
                           const IoletStep *io_dev = nullptr);

// The work list of a fused AA step pair (LBM_ORDER_SLABS): the bulk sites
// fall into chunks of whole z planes, each site's neighbours in its own or
// the two neighbouring chunks; an item is a run of at most 256 sites of one
// chunk and one of the two steps.  Items are listed chunk c's even runs, then
// chunk c - 2's odd runs, for c = 0 .. nchunks + 1, so every even run that an
// odd run depends on comes earlier in the list.  All device memory.
struct PairPlan {
    const int4 *items;  // {first site, end site, chunk, 1 for the odd step}
    int n_items;
    const int *tiles;   // [nchunks] even runs per chunk
    int nchunks;
    // [0] next item, [1] blocks finished, [2, 2 + nchunks) even runs done per
    // chunk; zero between launches (the last block to finish clears them)
    unsigned *ctr;
};

// An even AA step and the odd step after it in one pass over the bulk sites,
// by the plan W: A in natural layout on entry and exit.  io_dev_even /
// io_dev_odd, when not null, replace the iolet records.
cudaError_t launch_step_aa_pair(const DevLattice &L, void *A, const IoletStep &io_even, const IoletStep &io_odd,
                                cudaStream_t s, const IoletStep *io_dev_even, const IoletStep *io_dev_odd,
                                const PairPlan &W);

// The bounded waits of the step kernels, limit polls each, on a barrier no
// copy completes (bit 0 of *err when it gives up: the staged kernels'
// mbarrier wait) and on the counter *never, which nothing raises (bit 1: the
// fused step pair's counter wait).
cudaError_t launch_wait_probe(unsigned limit, int *err, const unsigned *never, cudaStream_t s);

// Exact copy of a stored state between layouts.
cudaError_t launch_relayout(const DevLattice &L, const void *src, int src_layout, void *dst,
                            int dst_layout, cudaStream_t s);

// rho, u, wss of the state held in f (any output may be null), caller order.
cudaError_t launch_macros(const DevLattice &L, const void *f, int layout, float *rho, float *u,
                          float *wss, cudaStream_t s);

// Deterministic float64 mass: partial sums into partials[nblk], final into out.
int mass_blocks();
cudaError_t launch_mass(const DevLattice &L, const void *f, int layout, double *partials, double *out,
                        cudaStream_t s);

// sum_x weight[x] q(x) of the state in f (q: 0 wall shear stress, 1
// density; weight float64 caller order or null), deterministic float64,
// through partials[mass_blocks()] into out.
cudaError_t launch_weighted_sum(const DevLattice &L, const void *f, int layout, int kind,
                                const double *weight, double *partials, double *out, cudaStream_t s);

// f(t) as float64 [q][n] caller order (gather of the stored state).
cudaError_t launch_gather_f64(const DevLattice &L, const void *f, int layout, double *out,
                              cudaStream_t s);
// stored state from float64 [q][n] caller order (inverse of the gather).
cudaError_t launch_scatter_f64(const DevLattice &L, const double *in, int layout, void *f,
                               cudaStream_t s);
// ------------------------------------------------------------ adjoint
// Per-step inputs of the adjoint kernel: the iolet densities of step t and
// the chain factors d rho_k / d amp = sin(2 pi t / T_k + phase_k) and
// d rho_k / d phase = amp_k cos(...), both 0 for a constant iolet.
struct AdjStep {
    IoletStep io;
    double dsin[kMaxIolets];
    double dacos[kMaxIolets];
};

// Objective term of one state f(t): when active, J += sum_x weight[x] q(x),
// q = wall shear stress (kind 0) or density (kind 1); weight is float64 in
// internal order; its state derivative enters the adjoint scaled by scale.
struct AdjObjective {
    int active;
    int kind;
    double scale;
    const double *weight;
    // float64 constants of tau, formed on the host (a float64 division per
    // site would load GB300's narrow FP64 pipe): 1/tau^2 and, for the wall
    // shear stress, d(ln coef)/dtau = (1/(2 tau^2)) / (1 - 1/(2 tau))
    double inv_tau2;
    double wss_dlog;
    // the same in float, for the per-site terms (summed per block in float,
    // then in float64 over blocks and steps)
    float inv_tau2_f, wss_dlog_f, scale_f;
};

int adjoint_blocks(const DevLattice &L);
// The adjoint of one AA step, in place on the one adjoint buffer lam: P is
// the stored state of time t in the AA form (natural layout: the adjoint of
// an even step, reading lam(t+1) in swapped form and writing lam(t) in site
// form; swapped layout: of an odd step, reading site form and writing
// swapped form); has_next = false for the terminal lam(T) (explicit terms
// only, written in the form the step t reads).  The bulk sites run on s, the
// sites with iolet links on t (t = s, or a stream forked from s and joined
// back by the caller: the two launches touch disjoint slots and accumulators).
cudaError_t launch_adjoint_aa(const DevLattice &L, const void *P, bool p_swapped, float *lam, bool has_next,
                              const AdjStep &st, const AdjObjective &obj, double *acc_block, double *io_acc,
                              cudaStream_t s, cudaStream_t t);
// One AA step from the state in src into dst (out of place: every slot of
// dst written), the layouts as for launch_step_aa.
cudaError_t launch_step_aa_oop(const DevLattice &L, const void *src, void *dst, bool odd, const IoletStep &io,
                               cudaStream_t s);
// lam_out = adjoint of step t at the state P = stored state of time t, from
// lam_next = lam(t+1) (null for the terminal state); accumulates J and
// dJ/dtau into acc_block[2 * blocks] and iolet derivatives into io_acc
// [3][n - n_bulk][q - 1].  Streams as for launch_adjoint_aa.
cudaError_t launch_adjoint(const DevLattice &L, const void *P, const float *lam_next, float *lam_out,
                           const AdjStep &st, const AdjObjective &obj, double *acc_block,
                           double *io_acc, cudaStream_t s, cudaStream_t t);
// out[0] = sum J, out[1] = dJ/dtau, out[2 + c * K + k] = iolet derivative c of iolet k
cudaError_t launch_adjoint_final(const DevLattice &L, const double *acc_block, const double *io_acc,
                                 double *out, cudaStream_t s);
// float32 site-form adjoint -> float64 [q][n] caller order
cudaError_t launch_lam_to_caller(const DevLattice &L, const float *lam, double *out, cudaStream_t s);

// Static float64 scratch of lbm_get_populations_noalloc (lbm_noalloc.cu):
// its capacity in values, and its device address on the current device
// (looked up on the first call per device).
size_t noalloc_max_values();
cudaError_t noalloc_scratch(double **out);

// ------------------------------------------------------------ rendering
// Where k_volume_fill writes: a float 3D surface of dims[0] x dims[1] x
// dims[2] voxels; a site at packed box coordinates p goes to voxel p + shift.
// quantity: 0 density, 1 speed |u|, 2 wall shear stress.  When mark is set,
// occ (bytes [bdims[2]][bdims[1]][bdims[0]], 8^3 bricks) is flagged where the
// voxel can reach a sample.
struct VolumeTarget {
    cudaSurfaceObject_t surf;
    int dims[3];
    int shift[3];
    int quantity;
    int mark;
    uint8_t *occ;
    int bdims[3];
};
cudaError_t launch_volume_fill(const DevLattice &L, const void *f, int layout, const uint64_t *vox,
                               const VolumeTarget &V, cudaStream_t s);

// Render parameters, float32, passed by value (the kernel keeps the view in
// the constant bank and copies the LUT into shared memory).
struct RenderArgs {
    float eye[3], fwd[3], right[3], up[3];
    float sx_mul, sy_mul;  // tan(fov_y / 2) W / H, tan(fov_y / 2)
    float dt, tf_scale, tf_offset, a_stop;
    int width, height;
    int dims[3];
    int bdims[3];
    int skip;    // skip bricks with occ == 0
    int filter;  // 0 texture-unit trilinear, 1 eight point fetches
    unsigned long long *counters;  // null, or [2]: += samples composited, brick jumps
    float lut[256][4];
};
// Ray-march the volume (tex_lin: linear filtering, tex_pt: point sampling,
// both unnormalised, clamped) into rgba [height][width][4]; dist is the
// brick distance map of launch_brick_distance.
cudaError_t launch_render(const RenderArgs &a, cudaTextureObject_t tex_lin, cudaTextureObject_t tex_pt,
                          const uint8_t *dist, float *rgba, cudaStream_t s);
// Chebyshev distance (in bricks, capped at 15) from every brick to the
// nearest flagged one, from the flags in marks (overwritten) into dist.
cudaError_t launch_brick_distance(uint8_t *marks, uint8_t *dist, const int (&bdims)[3], cudaStream_t s);
// Zero every voxel of a surface of dims.
cudaError_t launch_volume_clear(cudaSurfaceObject_t surf, const int (&dims)[3], cudaStream_t s);
// Brick occupancy of a dense float volume v [dims[2]][dims[1]][dims[0]]: occ
// must be zeroed; a brick is flagged when a non-zero voxel can reach it.
cudaError_t launch_occupancy(const float *v, const int (&dims)[3], uint8_t *occ, const int (&bdims)[3],
                             cudaStream_t s);

// stored state of the rest fluid (all deviations zero).
cudaError_t launch_zero(const DevLattice &L, void *f, cudaStream_t s);

}  // namespace hemelb_gb300
