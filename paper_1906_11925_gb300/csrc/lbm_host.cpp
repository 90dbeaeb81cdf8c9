// Host side of libhemelb_gb300: the C ABI declared in include/lbm.h.
//
// Set-up work (link building, validation, Morton reordering, folding of the
// link flags into the kernel table) runs here on the host in C++ with OpenMP;
// every per-step operation is a kernel launch on the context's stream.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lattice.h"
#include "lbm_internal.h"

#define HGB_API extern "C" __attribute__((visibility("default")))

namespace {
// NVTX range over one ABI call (visible to profilers that record NVTX, e.g.
// ncu --nvtx --nvtx-include); header-only NVTX, free when no tool is attached
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};
}  // namespace

using namespace hemelb_gb300;

// lbm_step's CUDA graphs: steps per captured chunk (even, so a chunk leaves
// the buffer roles and the AA layout as it found them) and pinned iolet
// record sets in flight
constexpr int kGraphSteps = 32;
// populations per slab chunk of the fused AA step pairs (LBM_ORDER_SLABS):
// the chunks between a chunk's even and odd step must stay in L2, and the
// lag (below) must exceed the sites that the resident blocks work on at once
// (608 blocks of 256), so that an odd run rarely waits; measured on the
// 10.8M-site tree, fp32: 1 MB with lag 14 306.6 us per step, 2 MB lag 6
// 309.8, 8 MB lag 2 311.3, 16 MB lag 2 327.1 (the unfused AA step 310.7)
#ifndef HGB_SLAB_BYTES
#define HGB_SLAB_BYTES (1 << 20)
#endif
constexpr int64_t kSlabBytes = HGB_SLAB_BYTES;
// sites per item of the fused pair's work list: one per thread of a block
constexpr int kPairRun = 256;
// chunks between a chunk's even runs and its odd runs in that list (>= 2)
#ifndef HGB_PAIR_LAG
#define HGB_PAIR_LAG 14
#endif
constexpr int kPairLag = HGB_PAIR_LAG;
static_assert(kPairLag >= 2, "an odd run needs the even runs of the next chunk done");
constexpr int kGraphRing = 8;
static_assert(kGraphSteps % 2 == 0, "a chunk must restore the buffer roles");

struct lbm_ctx {
    DevLattice L{};
    int q = 0;
    int storage = 0;
    int scale_log2 = 0;
    double tau = 0, rho0 = 1;
    int n_iolets = 0;
    int streaming = LBM_STREAM_PULL;
    bool aa_swapped = false;  // AA mode: the buffer holds the swapped layout
    int64_t n = 0, npad = 0;
    int64_t t = 0;
    cudaStream_t stream = nullptr;
    void *f_cur = nullptr, *f_nxt = nullptr;
    int32_t *tab = nullptr, *perm = nullptr;
    uint32_t *slots = nullptr;  // slot table of the bulk step kernels (see DevLattice::slots)
    // LBM_ORDER_SLABS with AA streaming: bounds of the slab chunks of the bulk
    // sites (empty: step pairs run unfused) and the fused pair's work list
    std::vector<int> slab_chunks;
    int4 *pair_items = nullptr;
    int *pair_tiles = nullptr;
    unsigned *pair_ctr = nullptr;
    PairPlan pair_plan{};
    double io_mean[LBM_MAX_IOLETS] = {}, io_amp[LBM_MAX_IOLETS] = {};
    double io_period[LBM_MAX_IOLETS] = {}, io_phase[LBM_MAX_IOLETS] = {};
    int io_kind[LBM_MAX_IOLETS] = {};
    double io_normal[LBM_MAX_IOLETS][3] = {};
    bool has_velocity_iolet = false;
    bool has_bfl = false;  // interpolated wall links in the table
    SideStream side{nullptr, nullptr, nullptr};  // for the launch after the bulk
    int *flags = nullptr;        // device: [0] instability check, [1] guard check
    cudaEvent_t handover = nullptr;  // lbm_set_stream: old stream -> new stream
    int64_t check_every = 0;     // lbm_set_stability_check (0: off)
    double check_umax = 0.3;
    // lbm_step's CUDA graphs (see run_graph_chunks): one captured chunk of
    // kGraphSteps steps per starting buffer / AA layout
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        void *f_cur = nullptr;
        bool swapped = false;
    };
    struct Graphs {
        GraphSlot slot[2];
        int evict = 0;
        IoletStep *io_dev = nullptr;  // [kGraphSteps] iolet records read by the replay
        IoletStep *io_pin = nullptr;  // [kGraphRing][kGraphSteps] pinned host records
        cudaEvent_t ring_ev[kGraphRing] = {};  // a ring slot's copy has been done
        int ring_next = 0;
        cudaStream_t cap = nullptr;   // capture stream
        bool off = false;             // set up failed or a capture failed: one launch per step
        bool ready = false;           // a step ran through the launchers (their one-time set-up)
    } graphs;
    float *vel_weight = nullptr;
    double *partials = nullptr, *mass_dev = nullptr;
    int *err_flag = nullptr;
    // a step kernel gave up waiting for its table copies (read back by
    // lbm_mass): the stored state is undefined until lbm_set_state or
    // lbm_set_populations replaces it, and the stepping calls refuse to run
    bool state_undefined = false;
    double *rho_io = nullptr;  // driven iolet densities, grown on demand
    size_t rho_io_cap = 0;
    double *mass_series = nullptr;
    size_t mass_series_cap = 0;
    size_t device_bytes = 0;
    std::vector<int32_t> perm_host;
    // adjoint workspace, kept between lbm_objective_grad calls (grown on demand)
    struct Workspace {
        std::vector<void *> slots;
        void *W0 = nullptr, *W1 = nullptr;  // W0: AA mode only
        float *lam[2] = {nullptr, nullptr};
        double *weight = nullptr, *acc_block = nullptr, *io_acc = nullptr, *out = nullptr;
        double *lam0 = nullptr;
        size_t bytes = 0;
        cudaEvent_t ev[2] = {nullptr, nullptr};
    } ws;
    int64_t last_fwd_steps = 0, last_adj_steps = 0;
    double last_sweep_ms = 0.0;
    // rendering: bounding box of the sites, their box coordinates packed 21
    // bits per axis in internal order (device copy made on first use), and a
    // serial number that tells volumes which lattice they hold
    int32_t box_lo[3] = {0, 0, 0}, box_dims[3] = {0, 0, 0};
    std::vector<uint64_t> vox_host;
    uint64_t *vox = nullptr;
    uint64_t serial = 0;
    std::string err;
};

struct lbm_volume {
    int dims[3] = {0, 0, 0};
    int bdims[3] = {0, 0, 0};
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex_lin = 0, tex_pt = 0;
    cudaSurfaceObject_t surf = 0;
    uint8_t *occ = nullptr;   // brick flags (scratch of the distance transform)
    uint8_t *dist = nullptr;  // brick distance map read by the render kernel
    size_t occ_bytes = 0;
    uint64_t lattice_serial = 0;  // lattice whose sites the volume holds (0: other content)
    int shift[3] = {0, 0, 0};
};

namespace {

thread_local std::string g_err;

lbm_status fail(lbm_ctx *ctx, lbm_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    g_err = msg;
    return st;
}

lbm_status cuda_fail(lbm_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, LBM_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, call)                                             \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

size_t elem_bytes(int storage) { return storage == LBM_STORE_FP32 ? 4 : 2; }

// ------------------------------------------------------------------ links

// Dense map of 8^3 voxel blocks over the bounding box of the site list; each
// occupied block stores the 512 site indices of its voxels (-1 = none).
class BlockMap {
   public:
    BlockMap(int64_t n, const int32_t *xyz) {
        if (n == 0) return;
        for (int a = 0; a < 3; ++a) {
            lo_[a] = xyz[a];
            hi_[a] = xyz[a];
        }
        for (int64_t x = 0; x < n; ++x)
            for (int a = 0; a < 3; ++a) {
                lo_[a] = std::min<int64_t>(lo_[a], xyz[3 * x + a]);
                hi_[a] = std::max<int64_t>(hi_[a], xyz[3 * x + a]);
            }
        for (int a = 0; a < 3; ++a) nb_[a] = ((hi_[a] - lo_[a]) >> 3) + 1;
        blocks_.assign((size_t)(nb_[0] * nb_[1] * nb_[2]), -1);
        for (int64_t x = 0; x < n; ++x) {
            int64_t b = block_of(xyz[3 * x], xyz[3 * x + 1], xyz[3 * x + 2]);
            if (blocks_[b] < 0) {
                blocks_[b] = (int64_t)(cells_.size() >> 9);
                cells_.resize(cells_.size() + 512, -1);
            }
        }
    }
    // insert site x; returns false if the voxel is already taken
    bool insert(int64_t x, const int32_t *p) {
        int32_t &c = cell(p[0], p[1], p[2]);
        if (c >= 0) return false;
        c = (int32_t)x;
        return true;
    }
    int32_t find(int64_t x, int64_t y, int64_t z) const {
        if (x < lo_[0] || y < lo_[1] || z < lo_[2] || x > hi_[0] || y > hi_[1] || z > hi_[2])
            return -1;
        int64_t b = blocks_[block_of(x, y, z)];
        if (b < 0) return -1;
        return cells_[(size_t)(b << 9) + local(x, y, z)];
    }

   private:
    int64_t block_of(int64_t x, int64_t y, int64_t z) const {
        return (((z - lo_[2]) >> 3) * nb_[1] + ((y - lo_[1]) >> 3)) * nb_[0] + ((x - lo_[0]) >> 3);
    }
    int64_t local(int64_t x, int64_t y, int64_t z) const {
        return (((z - lo_[2]) & 7) << 6) | (((y - lo_[1]) & 7) << 3) | ((x - lo_[0]) & 7);
    }
    int32_t &cell(int64_t x, int64_t y, int64_t z) {
        return cells_[(size_t)(blocks_[block_of(x, y, z)] << 9) + local(x, y, z)];
    }
    int64_t lo_[3] = {0, 0, 0}, hi_[3] = {-1, -1, -1}, nb_[3] = {0, 0, 0};
    std::vector<int64_t> blocks_;
    std::vector<int32_t> cells_;
};

inline int64_t vkey(int64_t x, int64_t y, int64_t z) {
    return ((z + (1LL << 20)) << 42) | ((y + (1LL << 20)) << 21) | (x + (1LL << 20));
}

// Morton (Z-order) key of a voxel, coordinates relative to the box minimum.
inline uint64_t spread3(uint64_t v) {
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}


// Iolet densities of step t: rho_k(t) = mean + amp sin(2 pi t / period + phase),
// in float64 on the host; the kernel receives rho_k and rho_k - rho0 as float.
// A velocity iolet carries its speed U_k(t) in rho[k] and its normal in nrm[k].
IoletStep iolet_step(const lbm_ctx *c, int64_t t) {
    IoletStep s{};
    for (int k = 0; k < c->n_iolets; ++k) {
        double r = c->io_mean[k];
        if (c->io_period[k] != 0.0 && c->io_amp[k] != 0.0)
            r += c->io_amp[k] * std::sin(2.0 * M_PI * (double)t / c->io_period[k] + c->io_phase[k]);
        s.drho[k] = (float)(r - c->rho0);
        s.rho[k] = (float)r;
        if (c->io_kind[k] == LBM_IOLET_VELOCITY) {
            s.vel_mask |= 1ull << k;
            for (int a = 0; a < 3; ++a) s.nrm[k][a] = (float)c->io_normal[k][a];
        }
    }
    return s;
}

// Layout of the current state buffer.
int cur_layout(const lbm_ctx *c) {
    if (c->streaming == LBM_STREAM_PULL) return LAYOUT_PULL;
    return c->aa_swapped ? LAYOUT_AA_SWAPPED : LAYOUT_NATURAL;
}

// The kinds of the iolets (velocity mask and normals) without their values:
// the record of the steps whose densities or speeds come from elsewhere.
IoletStep iolet_kinds(const lbm_ctx *c) {
    IoletStep s{};
    for (int k = 0; k < c->n_iolets; ++k)
        if (c->io_kind[k] == LBM_IOLET_VELOCITY) {
            s.vel_mask |= 1ull << k;
            for (int a = 0; a < 3; ++a) s.nrm[k][a] = (float)c->io_normal[k][a];
        }
    return s;
}

// One time step of the context's state (pull: two buffers; AA: in place).
// io_dev (device), when set, holds the step's iolet record in place of io.
cudaError_t advance_one(lbm_ctx *c, const IoletStep &io, const double *rho_io,
                        const IoletStep *io_dev = nullptr) {
    cudaError_t e;
    const SideStream *side = c->side.s ? &c->side : nullptr;
    if (c->streaming == LBM_STREAM_AA) {
        e = launch_step_aa(c->L, c->f_cur, c->aa_swapped, io, rho_io, c->stream, side, io_dev);
        if (e == cudaSuccess) c->aa_swapped = !c->aa_swapped;
    } else {
        e = launch_step(c->L, c->f_cur, c->f_nxt, io, rho_io, c->stream, side, io_dev);
        if (e == cudaSuccess) std::swap(c->f_cur, c->f_nxt);
    }
    return e;
}

// An even step and the odd step after it as one fused pass over the slab
// chunks (AA contexts in the LBM_ORDER_SLABS order, natural layout on entry);
// the same populations as two advance_one calls.
bool pairs_fused(const lbm_ctx *c) {
    return c->streaming == LBM_STREAM_AA && !c->slab_chunks.empty() && !c->aa_swapped;
}
cudaError_t advance_pair(lbm_ctx *c, const IoletStep &io_even, const IoletStep &io_odd,
                         const IoletStep *io_dev_even = nullptr, const IoletStep *io_dev_odd = nullptr) {
    return launch_step_aa_pair(c->L, c->f_cur, io_even, io_odd, c->stream, io_dev_even, io_dev_odd,
                               c->pair_plan);
}

// ---- CUDA graphs of lbm_step ----------------------------------------------
// lbm_step runs whole chunks of kGraphSteps steps as one replay of a captured
// CUDA graph: the same kernels with the same arguments as one launch per
// step, except that each step reads its iolet record (iolet_step, computed on
// the host as for a launch) from io_dev, which the host refills, stream-
// ordered, before every replay from a ring of pinned records.  The chunk is
// even, so it leaves the buffer roles (pull) and the layout (AA) as it found
// them; one graph is kept per starting buffer / layout.  On small lattices
// the per-launch host cost, not the kernels, sets the step rate.

void graphs_reset(lbm_ctx *c) {
    for (auto &g : c->graphs.slot) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = lbm_ctx::GraphSlot{};
    }
}

bool graphs_setup(lbm_ctx *c) {
    auto &G = c->graphs;
    if (G.io_dev) return true;
    cudaError_t e = cudaMalloc((void **)&G.io_dev, sizeof(IoletStep) * kGraphSteps);
    if (e == cudaSuccess)
        e = cudaMallocHost((void **)&G.io_pin, sizeof(IoletStep) * kGraphSteps * kGraphRing);
    for (int r = 0; r < kGraphRing && e == cudaSuccess; ++r)
        e = cudaEventCreateWithFlags(&G.ring_ev[r], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        G.off = true;
        return false;
    }
    return true;
}

// The graph of one chunk from the current buffer / layout (captured on first
// use), or null: the caller then launches step by step.
cudaGraphExec_t graph_for(lbm_ctx *c) {
    auto &G = c->graphs;
    for (auto &g : G.slot)
        if (g.exec && g.f_cur == c->f_cur && g.swapped == c->aa_swapped) return g.exec;
    if (!graphs_setup(c)) return nullptr;
    void *cur = c->f_cur, *nxt = c->f_nxt;
    const bool sw = c->aa_swapped;
    const cudaStream_t user = c->stream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    c->stream = G.cap;
    cudaError_t e = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        const IoletStep none{};
        for (int j = 0; j < kGraphSteps && e == cudaSuccess;) {
            if (pairs_fused(c) && j + 1 < kGraphSteps) {
                e = advance_pair(c, none, none, G.io_dev + j, G.io_dev + j + 1);
                j += 2;
            } else {
                e = advance_one(c, none, nullptr, G.io_dev + j);
                ++j;
            }
        }
        const cudaError_t e2 = cudaStreamEndCapture(G.cap, &graph);
        if (e == cudaSuccess) e = e2;
    }
    c->stream = user;
    c->f_cur = cur;
    c->f_nxt = nxt;
    c->aa_swapped = sw;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0ULL);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (exec) cudaGraphExecDestroy(exec);
        G.off = true;
        return nullptr;
    }
    auto &g = G.slot[G.evict];
    G.evict ^= 1;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = exec;
    g.f_cur = cur;
    g.swapped = sw;
    return exec;
}

// Whole chunks of the next `steps` steps as graph replays; returns the number
// of steps done (a multiple of kGraphSteps, 0 when graphs are not in use).
cudaError_t run_graph_chunks(lbm_ctx *c, int64_t steps, int64_t *done) {
    *done = 0;
    auto &G = c->graphs;
    if (G.off || !G.ready || c->n == 0 || steps < kGraphSteps) return cudaSuccess;
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &st) != cudaSuccess || st != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return cudaSuccess;  // the caller is capturing this stream itself
    }
    while (steps - *done >= kGraphSteps) {
        const cudaGraphExec_t exec = graph_for(c);
        if (!exec) return cudaSuccess;
        const int r = G.ring_next;
        G.ring_next = (r + 1) % kGraphRing;
        cudaError_t e = cudaEventSynchronize(G.ring_ev[r]);  // the ring slot's last copy is done
        if (e != cudaSuccess) return e;
        IoletStep *h = G.io_pin + (size_t)r * kGraphSteps;
        for (int j = 0; j < kGraphSteps; ++j) h[j] = iolet_step(c, c->t + j);
        e = cudaMemcpyAsync(G.io_dev, h, sizeof(IoletStep) * kGraphSteps, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(G.ring_ev[r], c->stream);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, c->stream);
        if (e != cudaSuccess) return e;
        c->t += kGraphSteps;
        *done += kGraphSteps;
    }
    return cudaSuccess;
}

}  // namespace

HGB_API const char *lbm_last_error(const lbm_ctx *ctx) {
    if (ctx) return ctx->err.c_str();
    return g_err.c_str();
}

HGB_API lbm_status lbm_links_build(int32_t q, int64_t n, const int32_t *xyz, int64_t n_io,
                                   const int32_t *io_xyz, const int32_t *io_id,
                                   const int32_t *periodic, int32_t *nbr, uint8_t *link) {
    if (q != 15 && q != 19) return fail(nullptr, LBM_ERR_ARG, "q must be 15 or 19");
    if (n < 0 || n_io < 0) return fail(nullptr, LBM_ERR_ARG, "negative size");
    if (n >= (1LL << 31) - 1024) return fail(nullptr, LBM_ERR_ARG, "too many sites");
    if (n > 0 && (!xyz || !nbr || !link)) return fail(nullptr, LBM_ERR_ARG, "NULL array");
    if (n_io > 0 && (!io_xyz || !io_id)) return fail(nullptr, LBM_ERR_ARG, "NULL iolet array");
    const int64_t lim = 1LL << 19;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (xyz[i] < -lim || xyz[i] >= lim) return fail(nullptr, LBM_ERR_ARG, "coordinate out of range");
    for (int64_t m = 0; m < n_io; ++m) {
        if (io_id[m] < 0 || io_id[m] >= LBM_MAX_IOLETS)
            return fail(nullptr, LBM_ERR_ARG, "iolet id out of range");
        for (int a = 0; a < 3; ++a)
            if (io_xyz[3 * m + a] < -lim || io_xyz[3 * m + a] >= lim)
                return fail(nullptr, LBM_ERR_ARG, "iolet coordinate out of range");
    }
    int32_t per[3] = {0, 0, 0};
    if (periodic)
        for (int a = 0; a < 3; ++a) {
            if (periodic[a] < 0) return fail(nullptr, LBM_ERR_ARG, "negative period");
            per[a] = periodic[a];
        }
    BlockMap map(n, xyz);
    for (int64_t x = 0; x < n; ++x)
        if (!map.insert(x, xyz + 3 * x)) return fail(nullptr, LBM_ERR_ARG, "duplicate fluid voxel");
    std::unordered_map<int64_t, int32_t> io;
    io.reserve((size_t)n_io * 2 + 1);
    for (int64_t m = 0; m < n_io; ++m) {
        int64_t k = vkey(io_xyz[3 * m], io_xyz[3 * m + 1], io_xyz[3 * m + 2]);
        auto it = io.find(k);
        if (it == io.end() || io_id[m] < it->second) io[k] = io_id[m];
    }
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < n; ++x) {
        for (int i = 0; i < q; ++i) {
            int64_t p[3];
            for (int a = 0; a < 3; ++a) {
                p[a] = (int64_t)xyz[3 * x + a] + cdir_q(q, i, a);
                if (per[a] > 0) p[a] = ((p[a] % per[a]) + per[a]) % per[a];
            }
            const int32_t j = map.find(p[0], p[1], p[2]);
            const int64_t o = (int64_t)i * n + x;
            if (j >= 0) {
                nbr[o] = j;
                link[o] = 0;
            } else {
                nbr[o] = -1;
                auto it = io.find(vkey(p[0], p[1], p[2]));
                link[o] = (uint8_t)(it == io.end() ? 1 : 2 + it->second);
            }
        }
    }
    return LBM_OK;
}

namespace {

lbm_status validate_params(const lbm_params *p) {
    if (!p) return fail(nullptr, LBM_ERR_ARG, "params is NULL");
    if (p->q != 15 && p->q != 19) return fail(nullptr, LBM_ERR_ARG, "q must be 15 or 19");
    if (p->storage != LBM_STORE_FP32 && p->storage != LBM_STORE_FP16 && p->storage != LBM_STORE_I16)
        return fail(nullptr, LBM_ERR_ARG, "storage must be LBM_STORE_FP32, LBM_STORE_FP16 or LBM_STORE_I16");
    if (!(p->tau > 0.5) || !std::isfinite(p->tau))
        return fail(nullptr, LBM_ERR_ARG, "tau must be finite and > 0.5");
    if (!(p->rho0 > 0) || !std::isfinite(p->rho0))
        return fail(nullptr, LBM_ERR_ARG, "rho0 must be finite and > 0");
    if (p->storage == LBM_STORE_FP16 && (p->fp16_scale_log2 < 0 || p->fp16_scale_log2 > 24))
        return fail(nullptr, LBM_ERR_ARG, "fp16_scale_log2 must be in [0, 24]");
    if (p->storage == LBM_STORE_I16 && (p->fp16_scale_log2 < 0 || p->fp16_scale_log2 > 30))
        return fail(nullptr, LBM_ERR_ARG, "the int16 scale (fp16_scale_log2) must be in [0, 30]");
    if (p->streaming != LBM_STREAM_PULL && p->streaming != LBM_STREAM_AA)
        return fail(nullptr, LBM_ERR_ARG, "streaming must be LBM_STREAM_PULL or LBM_STREAM_AA");
    if (p->site_order != LBM_ORDER_MORTON_RUNS && p->site_order != LBM_ORDER_MORTON &&
        p->site_order != LBM_ORDER_ROWS && p->site_order != LBM_ORDER_SLABS)
        return fail(nullptr, LBM_ERR_ARG, "unknown site_order");
    if (p->n_iolets < 0 || p->n_iolets > LBM_MAX_IOLETS)
        return fail(nullptr, LBM_ERR_ARG, "n_iolets out of range");
    if (p->n_iolets > 0 && (!p->rho_mean || !p->amp || !p->period || !p->phase))
        return fail(nullptr, LBM_ERR_ARG, "iolet arrays are NULL");
    for (int k = 0; k < p->n_iolets; ++k) {
        const int kind = p->iolet_kind ? p->iolet_kind[k] : LBM_IOLET_DENSITY;
        if (kind != LBM_IOLET_DENSITY && kind != LBM_IOLET_VELOCITY)
            return fail(nullptr, LBM_ERR_ARG, "iolet kind must be LBM_IOLET_DENSITY or LBM_IOLET_VELOCITY");
        if (!std::isfinite(p->rho_mean[k]) || !std::isfinite(p->amp[k]) || !std::isfinite(p->period[k]) ||
            p->period[k] < 0 || !std::isfinite(p->phase[k]))
            return fail(nullptr, LBM_ERR_ARG, "bad iolet schedule");
        if (kind == LBM_IOLET_DENSITY && !(p->rho_mean[k] > 0))
            return fail(nullptr, LBM_ERR_ARG, "bad iolet schedule");
        if (kind == LBM_IOLET_VELOCITY) {
            if (!p->iolet_normal) return fail(nullptr, LBM_ERR_ARG, "velocity iolet without a normal");
            const double *nv = p->iolet_normal + 3 * k;
            const double nn = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
            if (!std::isfinite(nn) || std::fabs(nn - 1.0) > 1e-6)
                return fail(nullptr, LBM_ERR_ARG, "velocity iolet normal must be a unit vector");
        }
    }
    return LBM_OK;
}

lbm_status validate_tables(int q, int n_iolets, int64_t n, const int32_t *nbr, const uint8_t *link) {
    int bad = 0;
    int64_t bad_x = -1, bad_i = -1;
#pragma omp parallel for schedule(static) reduction(max : bad)
    for (int64_t x = 0; x < n; ++x) {
        for (int i = 0; i < q; ++i) {
            const int64_t o = (int64_t)i * n + x;
            const int32_t nb = nbr[o];
            const int lk = link[o];
            int b = 0;
            if (i == 0) {
                b = (nb != x || lk != 0);
            } else if (lk == 0) {
                b = (nb < 0 || nb >= n) ? 1 : (nbr[(int64_t)opp(i) * n + nb] != x);
            } else if (lk == 1) {
                b = nb != -1;
            } else {
                b = (lk - 2 >= n_iolets) || nb != -1;
            }
            if (b) {
                bad = 1;
#pragma omp critical
                {
                    bad_x = x;
                    bad_i = i;
                }
            }
        }
    }
    if (bad) {
        char msg[160];
        snprintf(msg, sizeof msg,
                 "inconsistent link table at site %lld direction %lld (range, symmetry or flag)",
                 (long long)bad_x, (long long)bad_i);
        return fail(nullptr, LBM_ERR_TABLE, msg);
    }
    return LBM_OK;
}

void free_workspace(lbm_ctx *c) {
    auto &w = c->ws;
    for (void *p : w.slots) cudaFree(p);
    w.slots.clear();
    cudaFree(w.W0);
    cudaFree(w.W1);
    cudaFree(w.lam[0]);
    cudaFree(w.lam[1]);
    cudaFree(w.weight);
    cudaFree(w.acc_block);
    cudaFree(w.io_acc);
    cudaFree(w.out);
    cudaFree(w.lam0);
    for (auto &e : w.ev)
        if (e) cudaEventDestroy(e);
    c->device_bytes -= w.bytes;
    w = lbm_ctx::Workspace{};
}

void free_ctx(lbm_ctx *c) {
    if (!c) return;
    free_workspace(c);
    cudaFree(c->f_cur);
    cudaFree(c->f_nxt);
    cudaFree(c->tab);
    cudaFree(c->vel_weight);
    cudaFree(c->slots);
    cudaFree(c->pair_items);
    cudaFree(c->pair_tiles);
    cudaFree(c->pair_ctr);
    cudaFree(c->perm);
    cudaFree(c->partials);
    cudaFree(c->err_flag);
    cudaFree(c->mass_dev);
    cudaFree(c->rho_io);
    cudaFree(c->mass_series);
    cudaFree(c->vox);
    cudaFree(c->flags);
    if (c->side.s) cudaStreamDestroy(c->side.s);
    if (c->side.fork) cudaEventDestroy(c->side.fork);
    if (c->side.join) cudaEventDestroy(c->side.join);
    if (c->handover) cudaEventDestroy(c->handover);
    graphs_reset(c);
    cudaFree(c->graphs.io_dev);
    if (c->graphs.io_pin) cudaFreeHost(c->graphs.io_pin);
    for (cudaEvent_t ev : c->graphs.ring_ev)
        if (ev) cudaEventDestroy(ev);
    if (c->graphs.cap) cudaStreamDestroy(c->graphs.cap);
    delete c;
}

template <typename T>
cudaError_t dmalloc(lbm_ctx *c, T **p, size_t bytes) {
    cudaError_t e = cudaMalloc((void **)p, bytes ? bytes : 16);
    if (e == cudaSuccess) c->device_bytes += bytes;
    return e;
}

}  // namespace

HGB_API lbm_status lbm_create(lbm_ctx **out, const lbm_params *p, int64_t n, const int32_t *xyz,
                              const int32_t *nbr, const uint8_t *link, void *cuda_stream) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    const Range range("lbm_create");
    *out = nullptr;
    lbm_status st = validate_params(p);
    if (st != LBM_OK) return st;
    if (n < 0) return fail(nullptr, LBM_ERR_ARG, "negative n");
    if (n >= (1LL << 31) - 1024) return fail(nullptr, LBM_ERR_ARG, "too many sites");
    if (n > 0 && (!xyz || !nbr || !link)) return fail(nullptr, LBM_ERR_ARG, "NULL array");
    const int q = p->q;
    // the kernels address a population plane slot as a 32-bit offset
    const int64_t npad = std::max<int64_t>(128, (n + 127) / 128 * 128);
    if ((int64_t)q * npad >= (1LL << 31))
        return fail(nullptr, LBM_ERR_ARG, "too many sites: q * npad must stay below 2^31");
    st = validate_tables(q, p->n_iolets, n, nbr, link);
    if (st != LBM_OK) return st;
    // interpolated walls: q in (0, 1] on every wall link
    const double *wq = p->wall_q;
    bool any_bfl = false;
    if (wq) {
        for (int64_t o = 0; o < (int64_t)q * n; ++o) {
            if (link[o] != 1) continue;
            if (!(wq[o] > 0.0 && wq[o] <= 1.0)) return fail(nullptr, LBM_ERR_ARG, "wall_q must lie in (0, 1]");
            any_bfl |= wq[o] != 0.5;
        }
    }
    auto bfl_link = [&](int64_t o) { return any_bfl && link[o] == 1 && wq[o] != 0.5; };
    const int64_t lim = 1LL << 19;
    for (int64_t i = 0; i < 3 * n; ++i)
        if (xyz[i] < -lim || xyz[i] >= lim) return fail(nullptr, LBM_ERR_ARG, "coordinate out of range");

    const size_t eb = elem_bytes(p->storage);
    const size_t nbuf = p->streaming == LBM_STREAM_AA ? 1 : 2;
    // populations, the pull-source table, the slot table of the bulk sites,
    // the permutation and the reduction scratch
    const size_t need = nbuf * ((size_t)q * npad + (size_t)kGuardSlots) * eb + 2 * (size_t)(q - 1) * npad * 4 +
                        (size_t)n * 4 + (size_t)(mass_blocks() + 8) * 8;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaMemGetInfo");
    if (need + (64u << 20) > free_b) {
        char msg[160];
        snprintf(msg, sizeof msg, "need %zu bytes of device memory, %zu free", need, free_b);
        return fail(nullptr, LBM_ERR_NOMEM, msg);
    }

    // Internal order: sites without iolet links along the chosen curve
    // (site_order), then the sites with an iolet link along it (the kernel tests x >= n_bulk
    // instead of scanning the table for iolet entries).
    std::vector<int32_t> perm((size_t)n);
    int64_t n_bulk = 0;
    {
        int64_t lo[3] = {0, 0, 0};
        if (n > 0)
            for (int a = 0; a < 3; ++a) {
                lo[a] = xyz[a];
                for (int64_t x = 0; x < n; ++x) lo[a] = std::min<int64_t>(lo[a], xyz[3 * x + a]);
            }
        std::vector<std::pair<uint64_t, int32_t>> keys((size_t)n);
#pragma omp parallel for schedule(static) reduction(+ : n_bulk)
        for (int64_t x = 0; x < n; ++x) {
            const uint64_t rx = (uint64_t)(xyz[3 * x] - lo[0]), ry = (uint64_t)(xyz[3 * x + 1] - lo[1]),
                           rz = (uint64_t)(xyz[3 * x + 2] - lo[2]);
            bool io_site = false;  // an iolet or an interpolated wall link
            for (int i = 1; i < q; ++i)
                io_site |= link[(int64_t)i * n + x] >= 2 || bfl_link((int64_t)i * n + x);
            // the sites after the bulk lie on the walls and iolets (a shell,
            // not runs along x): they keep the plain Morton order
            uint64_t k;
            if (p->site_order == LBM_ORDER_ROWS || p->site_order == LBM_ORDER_SLABS)
                k = (rz << 42) | (ry << 21) | rx;
            else if (p->site_order == LBM_ORDER_MORTON_RUNS && !io_site)
                k = ((spread3(rx >> 5) | (spread3(ry) << 1) | (spread3(rz) << 2)) << 5) | (rx & 31);
            else
                k = spread3(rx) | (spread3(ry) << 1) | (spread3(rz) << 2);
            if (!io_site) ++n_bulk;
            keys[(size_t)x] = {k | ((uint64_t)io_site << 63), (int32_t)x};
        }
        std::sort(keys.begin(), keys.end());
        for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = keys[(size_t)i].second;
    }
    std::vector<int32_t> inv((size_t)n);
    for (int64_t i = 0; i < n; ++i) inv[(size_t)perm[(size_t)i]] = (int32_t)i;

    // kernel table: pull source of population i at internal site xi
    std::vector<int32_t> tab((size_t)(q - 1) * npad, 0);
#pragma omp parallel for schedule(static)
    for (int64_t xi = 0; xi < n; ++xi) {
        const int64_t x = perm[(size_t)xi];
        for (int i = 1; i < q; ++i) {
            const int j = opp(i);  // the link that population i arrives through
            const int lk = link[(int64_t)j * n + x];
            tab[(size_t)(i - 1) * npad + xi] = lk == 0 ? inv[(size_t)nbr[(int64_t)j * n + x]]
                                               : bfl_link((int64_t)j * n + x) ? bfl_code(wq[(int64_t)j * n + x])
                                                                              : -lk;
        }
    }

    // slot table of the bulk sites: the element offset, in the population
    // buffer, that the bulk step kernel reads population i of site xi from
    // (pull: the pull source's slot; AA: the slot the odd step reads and
    // writes back), so that those kernels do no address arithmetic beyond one
    // multiply-add per population
    std::vector<uint32_t> slots((size_t)(q - 1) * npad, 0);
    {
        const bool aa = p->streaming == LBM_STREAM_AA;
#pragma omp parallel for schedule(static)
        for (int64_t xi = 0; xi < n_bulk; ++xi)
            for (int i = 1; i < q; ++i) {
                const int32_t s = tab[(size_t)(i - 1) * npad + xi];
                const int64_t e = s >= 0 ? (int64_t)(aa ? opp(i) : i) * npad + s
                                         : (int64_t)(aa ? i : opp(i)) * npad + xi;
                slots[(size_t)(i - 1) * npad + xi] = (uint32_t)e;
            }
    }

    // slab chunks of the fused AA step pairs (LBM_ORDER_SLABS): runs of whole
    // z planes of the bulk sites, about kSlabBytes of populations each; kept
    // only if every fluid neighbour of a chunk's bulk sites lies in the chunk
    // or the two next to it (a periodic z axis, for instance, breaks that:
    // the pairs then run unfused)
    std::vector<int> slab_chunks;
    if (p->site_order == LBM_ORDER_SLABS && p->streaming == LBM_STREAM_AA && n_bulk > 0) {
        const int64_t target = std::max<int64_t>(4096, kSlabBytes / ((int64_t)q * (int64_t)eb));
        std::vector<int> chunk_of((size_t)n_bulk);
        slab_chunks.push_back(0);
        int32_t zprev = xyz[3 * (int64_t)perm[0] + 2];
        for (int64_t xi = 0; xi < n_bulk; ++xi) {
            const int32_t z = xyz[3 * (int64_t)perm[(size_t)xi] + 2];
            if (z != zprev && xi - slab_chunks.back() >= target) slab_chunks.push_back((int)xi);
            zprev = z;
            chunk_of[(size_t)xi] = (int)slab_chunks.size() - 1;
        }
        slab_chunks.push_back((int)n_bulk);
        bool ok = slab_chunks.size() >= 3;  // at least two chunks, or nothing to gain
#pragma omp parallel for schedule(static) reduction(&& : ok)
        for (int64_t xi = 0; xi < n_bulk; ++xi)
            for (int i = 1; i < q; ++i) {
                const int32_t src = tab[(size_t)(i - 1) * npad + xi];
                if (src >= 0 && src < n_bulk && std::abs(chunk_of[(size_t)src] - chunk_of[(size_t)xi]) > 1)
                    ok = false;
            }
        if (!ok) slab_chunks.clear();
    }

    lbm_ctx *c = new lbm_ctx();
    c->q = q;
    c->storage = p->storage;
    c->scale_log2 = p->storage == LBM_STORE_FP32 ? 0 : p->fp16_scale_log2;
    c->tau = p->tau;
    c->rho0 = p->rho0;
    c->n_iolets = p->n_iolets;
    c->streaming = p->streaming;
    c->n = n;
    c->npad = npad;
    c->stream = (cudaStream_t)cuda_stream;
    for (int k = 0; k < p->n_iolets; ++k) {
        c->io_mean[k] = p->rho_mean[k];
        c->io_amp[k] = p->amp[k];
        c->io_period[k] = p->period[k];
        c->io_phase[k] = p->phase[k];
        c->io_kind[k] = p->iolet_kind ? p->iolet_kind[k] : LBM_IOLET_DENSITY;
        if (c->io_kind[k] == LBM_IOLET_VELOCITY) {
            c->has_velocity_iolet = true;
            for (int a = 0; a < 3; ++a) c->io_normal[k][a] = p->iolet_normal[3 * k + a];
        }
    }
#define CKC(call)                                   \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) {                    \
            lbm_status s_ = cuda_fail(nullptr, e_, #call); \
            free_ctx(c);                            \
            return s_;                              \
        }                                           \
    } while (0)
    const size_t fbytes = ((size_t)q * npad + (size_t)kGuardSlots) * eb;  // planes + guard row
    CKC(dmalloc(c, &c->f_cur, fbytes));
    CKC(dmalloc(c, &c->flags, 16));
    if (c->streaming == LBM_STREAM_PULL) CKC(dmalloc(c, &c->f_nxt, fbytes));
    CKC(dmalloc(c, &c->tab, tab.size() * 4));
    CKC(dmalloc(c, &c->slots, slots.size() * 4));
    CKC(dmalloc(c, &c->perm, (size_t)n * 4));
    {
        // velocity-iolet weights of the iolet sites, internal order
        std::vector<float> wt((size_t)std::max<int64_t>(n - n_bulk, 1), 1.0f);
        if (p->velocity_weight)
            for (int64_t xi = n_bulk; xi < n; ++xi)
                wt[(size_t)(xi - n_bulk)] = (float)p->velocity_weight[perm[(size_t)xi]];
        CKC(dmalloc(c, &c->vel_weight, wt.size() * 4));
        CKC(cudaMemcpyAsync(c->vel_weight, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice, c->stream));
        CKC(cudaStreamSynchronize(c->stream));  // wt dies at the end of this block
    }
    CKC(dmalloc(c, &c->partials, (size_t)mass_blocks() * 8));
    CKC(dmalloc(c, &c->mass_dev, 8));
    CKC(dmalloc(c, &c->err_flag, 16));
    CKC(cudaMemsetAsync(c->err_flag, 0, 16, c->stream));
    CKC(cudaMemcpyAsync(c->tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CKC(cudaMemcpyAsync(c->slots, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice, c->stream));
    if (n) CKC(cudaMemcpyAsync(c->perm, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, c->stream));
    DevLattice &L = c->L;
    L.q = q;
    L.storage = p->storage;
    L.n = (int)n;
    L.n_bulk = (int)n_bulk;
    L.npad = npad;
    L.omega = (float)(1.0 / p->tau);
    L.tau = (float)p->tau;
    L.rho0 = (float)p->rho0;
    L.scale = (float)std::ldexp(1.0, c->scale_log2);
    L.inv_scale = (float)std::ldexp(1.0, -c->scale_log2);
    L.n_iolets = p->n_iolets;
    L.tab = c->tab;
    L.perm = c->perm;
    L.err = c->err_flag;
    L.vel_weight = c->vel_weight;
    L.slots = c->slots;
    L.bfl = any_bfl ? 1 : 0;
    c->has_bfl = any_bfl;
    if (n_bulk > 0 && n_bulk < n) {
        // the launch of the sites after the bulk runs beside the bulk launch
        CKC(cudaStreamCreateWithFlags(&c->side.s, cudaStreamNonBlocking));
        CKC(cudaEventCreateWithFlags(&c->side.fork, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&c->side.join, cudaEventDisableTiming));
    }
    CKC(launch_zero(L, c->f_cur, c->stream));
    if (c->f_nxt) CKC(launch_zero(L, c->f_nxt, c->stream));
    CKC(launch_guards(L, c->f_cur, false, nullptr, c->stream));
    if (c->f_nxt) CKC(launch_guards(L, c->f_nxt, false, nullptr, c->stream));
    CKC(cudaMemsetAsync(c->flags, 0, 16, c->stream));
    CKC(cudaStreamSynchronize(c->stream));  // host vectors die at return
#undef CKC
    if (!slab_chunks.empty()) {
        // the fused pair's work list: runs of up to kPairRun sites, chunk c's
        // even runs, then chunk (c - kPairLag)'s odd runs, for c = 0 ..
        // K + kPairLag - 1
        const int K = (int)slab_chunks.size() - 1;
        std::vector<int4> items;
        std::vector<int> tiles((size_t)K);
        auto runs = [&](int c, int odd) {
            for (int a = slab_chunks[(size_t)c]; a < slab_chunks[(size_t)c + 1]; a += kPairRun)
                items.push_back(make_int4(a, std::min(a + kPairRun, slab_chunks[(size_t)c + 1]), c, odd));
        };
        for (int c = 0; c < K + kPairLag; ++c) {
            if (c < K) {
                const size_t before = items.size();
                runs(c, 0);
                tiles[(size_t)c] = (int)(items.size() - before);
            }
            if (c >= kPairLag) runs(c - kPairLag, 1);
        }
        const size_t ctr_bytes = sizeof(unsigned) * (size_t)(2 + K);
        if (cudaMalloc((void **)&c->pair_items, sizeof(int4) * items.size()) != cudaSuccess ||
            cudaMalloc((void **)&c->pair_tiles, sizeof(int) * tiles.size()) != cudaSuccess ||
            cudaMalloc((void **)&c->pair_ctr, ctr_bytes) != cudaSuccess ||
            cudaMemcpy(c->pair_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(c->pair_tiles, tiles.data(), sizeof(int) * tiles.size(), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemset(c->pair_ctr, 0, ctr_bytes) != cudaSuccess) {
            cudaGetLastError();
            free_ctx(c);
            return fail(nullptr, LBM_ERR_CUDA, "allocation of the fused step pair's work list failed");
        }
        c->pair_plan = PairPlan{c->pair_items, (int)items.size(), c->pair_tiles, K, c->pair_ctr};
    }
    c->perm_host.swap(perm);
    c->slab_chunks.swap(slab_chunks);
    {
        static std::atomic<uint64_t> next_serial{0};
        c->serial = ++next_serial;
        int64_t lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
        if (n > 0)
            for (int a = 0; a < 3; ++a) {
                lo[a] = hi[a] = xyz[a];
                for (int64_t x = 0; x < n; ++x) {
                    lo[a] = std::min<int64_t>(lo[a], xyz[3 * x + a]);
                    hi[a] = std::max<int64_t>(hi[a], xyz[3 * x + a]);
                }
            }
        for (int a = 0; a < 3; ++a) {
            c->box_lo[a] = (int32_t)lo[a];
            c->box_dims[a] = (int32_t)(hi[a] - lo[a] + 1);
        }
        c->vox_host.resize((size_t)n);
        for (int64_t xi = 0; xi < n; ++xi) {
            const int64_t x = c->perm_host[(size_t)xi];
            c->vox_host[(size_t)xi] = (uint64_t)(xyz[3 * x] - lo[0]) |
                                      ((uint64_t)(xyz[3 * x + 1] - lo[1]) << 21) |
                                      ((uint64_t)(xyz[3 * x + 2] - lo[2]) << 42);
        }
    }
    *out = c;
    return LBM_OK;
}

HGB_API void lbm_destroy(lbm_ctx *ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
}

HGB_API lbm_status lbm_set_stream(lbm_ctx *ctx, void *cuda_stream) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    const cudaStream_t next = (cudaStream_t)cuda_stream;
    if (next != ctx->stream) {
        // the new stream waits for the work already queued on the old one
        if (!ctx->handover) CK(ctx, cudaEventCreateWithFlags(&ctx->handover, cudaEventDisableTiming));
        CK(ctx, cudaEventRecord(ctx->handover, ctx->stream));
        CK(ctx, cudaStreamWaitEvent(next, ctx->handover, 0));
    }
    ctx->stream = next;
    return LBM_OK;
}

namespace {
// nsteps steps: whole graph chunks, then one launch per step
lbm_status run_steps(lbm_ctx *ctx, int64_t nsteps) {
    if (ctx->state_undefined)
        return fail(ctx, LBM_ERR_STATE, "the state is undefined after a failed step; replace it with "
                    "lbm_set_state or lbm_set_populations");
    int64_t s = 0;
    if (nsteps > 0 && !ctx->graphs.ready) {
        // the first step goes through the launchers directly (their one-time
        // set-up must not happen inside a capture)
        CK(ctx, advance_one(ctx, iolet_step(ctx, ctx->t), nullptr));
        ++ctx->t;
        ctx->graphs.ready = true;
        s = 1;
    }
    int64_t done = 0;
    CK(ctx, run_graph_chunks(ctx, nsteps - s, &done));
    for (s += done; s < nsteps; ++s) {
        CK(ctx, advance_one(ctx, iolet_step(ctx, ctx->t), nullptr));
        ++ctx->t;
    }
    return LBM_OK;
}
}  // namespace

HGB_API lbm_status lbm_step(lbm_ctx *ctx, int64_t nsteps) {
    const Range range("lbm_step");
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, LBM_ERR_ARG, "nsteps < 0");
    const int64_t every = ctx->check_every;
    if (every <= 0 || nsteps == 0) return run_steps(ctx, nsteps);
    // checked: a check after every `every` steps and after the last; check j
    // (1-based) covers the steps up to t0 + min(j every, nsteps)
    const int64_t t0 = ctx->t;
    CK(ctx, cudaMemsetAsync(ctx->flags, 0, 4, ctx->stream));
    int64_t done = 0, j = 0;
    while (done < nsteps) {
        const int64_t m = std::min(every, nsteps - done);
        const lbm_status st = run_steps(ctx, m);
        if (st != LBM_OK) return st;
        done += m;
        ++j;
        const int tag = (int)std::min<int64_t>(j, INT32_MAX);
        CK(ctx, launch_stability(ctx->L, ctx->f_cur, (float)ctx->check_umax, tag, ctx->flags, ctx->stream));
    }
    int h = 0;
    CK(ctx, cudaMemcpyAsync(&h, ctx->flags, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (h > 0) {
        const int64_t lo = t0 + std::min((int64_t)(h - 1) * every, nsteps);
        const int64_t hi = h == INT32_MAX ? t0 + nsteps : t0 + std::min((int64_t)h * every, nsteps);
        char msg[200];
        snprintf(msg, sizeof msg,
                 "unstable: a stored value is not finite, or rho <= 0 or |u| > %g at a site, after the "
                 "steps of times %lld .. %lld",
                 ctx->check_umax, (long long)lo, (long long)(hi - 1));
        return fail(ctx, LBM_ERR_UNSTABLE, msg);
    }
    return LBM_OK;
}

HGB_API lbm_status lbm_set_stability_check(lbm_ctx *ctx, int64_t every, double u_max) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (every < 0) return fail(ctx, LBM_ERR_ARG, "every < 0");
    if (!(u_max > 0) || !std::isfinite(u_max)) return fail(ctx, LBM_ERR_ARG, "u_max must be finite and > 0");
    ctx->check_every = every;
    ctx->check_umax = u_max;
    return LBM_OK;
}

HGB_API lbm_status lbm_check_guards(lbm_ctx *ctx, int32_t *intact) {
    if (!ctx || !intact) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    CK(ctx, cudaMemsetAsync(ctx->flags + 1, 0, 4, ctx->stream));
    CK(ctx, launch_guards(ctx->L, ctx->f_cur, true, ctx->flags + 1, ctx->stream));
    if (ctx->f_nxt) CK(ctx, launch_guards(ctx->L, ctx->f_nxt, true, ctx->flags + 1, ctx->stream));
    int h = 0;
    CK(ctx, cudaMemcpyAsync(&h, ctx->flags + 1, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    *intact = h == 0 ? 1 : 0;
    return LBM_OK;
}

HGB_API lbm_status lbm_step_driven(lbm_ctx *ctx, int64_t nsteps, const double *rho_io_host,
                                   double *mass_host) {
    const Range range("lbm_step_driven");
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, LBM_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return LBM_OK;
    if (ctx->state_undefined)
        return fail(ctx, LBM_ERR_STATE, "the state is undefined after a failed step; replace it with "
                    "lbm_set_state or lbm_set_populations");
    const int K = ctx->n_iolets;
    if (K > 0 && !rho_io_host) return fail(ctx, LBM_ERR_ARG, "rho_io_host is NULL");
    const size_t need = (size_t)nsteps * (size_t)std::max(K, 1) * 8;
    if (need > ctx->rho_io_cap) {
        cudaFree(ctx->rho_io);
        ctx->rho_io = nullptr;
        ctx->rho_io_cap = 0;
        CK(ctx, cudaMalloc((void **)&ctx->rho_io, need));
        ctx->rho_io_cap = need;
    }
    if (mass_host && (size_t)nsteps * 8 > ctx->mass_series_cap) {
        cudaFree(ctx->mass_series);
        ctx->mass_series = nullptr;
        ctx->mass_series_cap = 0;
        CK(ctx, cudaMalloc((void **)&ctx->mass_series, (size_t)nsteps * 8));
        ctx->mass_series_cap = (size_t)nsteps * 8;
    }
    if (K > 0)
        CK(ctx, cudaMemcpyAsync(ctx->rho_io, rho_io_host, (size_t)nsteps * K * 8,
                                cudaMemcpyHostToDevice, ctx->stream));
    const IoletStep kinds = iolet_kinds(ctx);  // velocity iolets take the driven values as speeds
    for (int64_t s = 0; s < nsteps; ++s) {
        CK(ctx, advance_one(ctx, kinds, ctx->rho_io + s * K));
        ++ctx->t;
        if (mass_host)
            CK(ctx, launch_mass(ctx->L, ctx->f_cur, cur_layout(ctx), ctx->partials, ctx->mass_series + s, ctx->stream));
    }
    if (mass_host)
        CK(ctx, cudaMemcpyAsync(mass_host, ctx->mass_series, (size_t)nsteps * 8,
                                cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (mass_host)
        for (int64_t s = 0; s < nsteps; ++s)
            if (!std::isfinite(mass_host[s])) return fail(ctx, LBM_ERR_UNSTABLE, "non-finite mass");
    return LBM_OK;
}

HGB_API lbm_status lbm_get_time(const lbm_ctx *ctx, int64_t *t) {
    if (!ctx || !t) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    *t = ctx->t;
    return LBM_OK;
}

HGB_API lbm_status lbm_set_time(lbm_ctx *ctx, int64_t t) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (t < 0) return fail(ctx, LBM_ERR_ARG, "t < 0");
    ctx->t = t;
    return LBM_OK;
}

HGB_API lbm_status lbm_macros(lbm_ctx *ctx, float *rho_d, float *u_d, float *wss_d) {
    const Range range("lbm_macros");
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    CK(ctx, launch_macros(ctx->L, ctx->f_cur, cur_layout(ctx), rho_d, u_d, wss_d, ctx->stream));
    return LBM_OK;
}

HGB_API lbm_status lbm_mass(lbm_ctx *ctx, double *out) {
    if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    int flag = 0;
    CK(ctx, launch_mass(ctx->L, ctx->f_cur, cur_layout(ctx), ctx->partials, ctx->mass_dev, ctx->stream));
    CK(ctx, cudaMemcpyAsync(out, ctx->mass_dev, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaMemcpyAsync(&flag, ctx->err_flag, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag) ctx->state_undefined = true;
    if (flag == 2)
        return fail(ctx, LBM_ERR_CUDA, "a step kernel read a table entry out of range (checked build); the state "
                    "is undefined until lbm_set_state or lbm_set_populations");
    if (flag)
        return fail(ctx, LBM_ERR_CUDA, "a step kernel gave up waiting for its table copies; the state is "
                    "undefined until lbm_set_state or lbm_set_populations");
    if (!std::isfinite(*out)) return fail(ctx, LBM_ERR_UNSTABLE, "non-finite mass");
    return LBM_OK;
}

HGB_API lbm_status lbm_check_wait_timeout(uint32_t limit, void *cuda_stream, int32_t *gave_up) {
    if (!gave_up) return fail(nullptr, LBM_ERR_ARG, "gave_up is NULL");
    if (limit < 1 || limit > (1u << 24)) return fail(nullptr, LBM_ERR_ARG, "limit must lie in [1, 2^24]");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    int *flag = nullptr;  // [0] the probe's flag bits, [1] a counter nothing raises
    cudaError_t e = cudaMalloc((void **)&flag, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = launch_wait_probe(limit, flag, (const unsigned *)(flag + 1), s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lbm_check_wait_timeout");
    *gave_up = h == 3 ? 1 : 0;  // both waits gave up
    return LBM_OK;
}

HGB_API lbm_status lbm_weighted_sum(lbm_ctx *ctx, int32_t kind, const double *weight_d, double *out) {
    if (!ctx || !out) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (kind != LBM_OBJ_WSS && kind != LBM_OBJ_DENSITY) return fail(ctx, LBM_ERR_ARG, "unknown kind");
    CK(ctx, launch_weighted_sum(ctx->L, ctx->f_cur, cur_layout(ctx), kind == LBM_OBJ_DENSITY ? 1 : 0,
                                weight_d, ctx->partials, ctx->mass_dev, ctx->stream));
    CK(ctx, cudaMemcpyAsync(out, ctx->mass_dev, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (!std::isfinite(*out)) return fail(ctx, LBM_ERR_UNSTABLE, "non-finite sum");
    return LBM_OK;
}

HGB_API lbm_status lbm_get_populations(lbm_ctx *ctx, double *f_host) {
    if (!ctx || (!f_host && ctx->n)) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (ctx->n == 0) return LBM_OK;
    const size_t bytes = (size_t)ctx->q * ctx->n * 8;
    double *tmp = nullptr;
    CK(ctx, cudaMalloc((void **)&tmp, bytes));
    cudaError_t e = launch_gather_f64(ctx->L, ctx->f_cur, cur_layout(ctx), tmp, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f_host, tmp, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_get_populations");
    return LBM_OK;
}

HGB_API lbm_status lbm_set_populations(lbm_ctx *ctx, const double *f_host) {
    if (!ctx || (!f_host && ctx->n)) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (ctx->n == 0) return LBM_OK;
    {
        // every value finite and its deviation representable in the storage
        const double lim = ctx->storage == LBM_STORE_FP16 ? 65504.0 / std::ldexp(1.0, ctx->scale_log2)
                           : ctx->storage == LBM_STORE_I16 ? 32766.0 / std::ldexp(1.0, ctx->scale_log2)
                                                           : 3.4028234663852886e38;
        for (int i = 0; i < ctx->q; ++i) {
            const double w = wdir_q(ctx->q, i) * ctx->rho0;
            const double *row = f_host + (size_t)i * ctx->n;
            for (int64_t x = 0; x < ctx->n; ++x)
                if (!(std::fabs(row[x] - w) <= lim)) {
                    char msg[160];
                    snprintf(msg, sizeof msg, "population %d of site %lld is %g: not finite or out of the "
                             "storage range", i, (long long)x, row[x]);
                    return fail(ctx, LBM_ERR_UNSTABLE, msg);
                }
        }
    }
    const size_t bytes = (size_t)ctx->q * ctx->n * 8;
    double *tmp = nullptr;
    CK(ctx, cudaMalloc((void **)&tmp, bytes));
    cudaError_t e = cudaMemcpyAsync(tmp, f_host, bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = launch_scatter_f64(ctx->L, tmp, cur_layout(ctx), ctx->f_cur, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->err_flag, 0, 4, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_set_populations");
    ctx->state_undefined = false;
    return LBM_OK;
}

HGB_API lbm_status lbm_get_populations_noalloc(lbm_ctx *ctx, double *f_host) {
    if (!ctx || (!f_host && ctx->n)) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    const size_t count = (size_t)ctx->q * (size_t)ctx->n;
    if (count > noalloc_max_values()) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "lbm_get_populations_noalloc: q*n = %zu values exceeds the static scratch of "
                 "%zu float64 values; use lbm_get_populations",
                 count, noalloc_max_values());
        return fail(ctx, LBM_ERR_ARG, msg);
    }
    if (count == 0) return LBM_OK;
    {
        // a host copy and a stream synchronisation cannot be part of a capture
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        CK(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
        if (cs != cudaStreamCaptureStatusNone)
            return fail(ctx, LBM_ERR_STATE, "lbm_get_populations_noalloc: the context's stream is being captured");
    }
    // the scratch address is per device: look it up with the context's device current
    cudaPointerAttributes at{};
    CK(ctx, cudaPointerGetAttributes(&at, ctx->f_cur));
    int prev = 0;
    CK(ctx, cudaGetDevice(&prev));
    if (prev != at.device) CK(ctx, cudaSetDevice(at.device));
    double *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e == cudaSuccess) e = launch_gather_f64(ctx->L, ctx->f_cur, cur_layout(ctx), scratch, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f_host, scratch, count * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (prev != at.device) cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_get_populations_noalloc");
    return LBM_OK;
}

// The state blob is the raw stored buffer followed by an 8-byte trailer that
// records the AA layout phase (always 0 for pull streaming).
HGB_API lbm_status lbm_state_bytes(const lbm_ctx *ctx, size_t *bytes) {
    if (!ctx || !bytes) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    *bytes = (size_t)ctx->q * ctx->npad * elem_bytes(ctx->storage) + 8;
    return LBM_OK;
}

HGB_API lbm_status lbm_get_state(lbm_ctx *ctx, void *host, size_t bytes) {
    if (!ctx || !host) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    const size_t raw = (size_t)ctx->q * ctx->npad * elem_bytes(ctx->storage);
    if (bytes != raw + 8) return fail(ctx, LBM_ERR_ARG, "wrong state size");
    CK(ctx, cudaMemcpyAsync(host, ctx->f_cur, raw, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t phase = ctx->aa_swapped ? 1 : 0;
    memcpy(static_cast<char *>(host) + raw, &phase, 8);
    return LBM_OK;
}

HGB_API lbm_status lbm_set_state(lbm_ctx *ctx, const void *host, size_t bytes) {
    if (!ctx || !host) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    const size_t raw = (size_t)ctx->q * ctx->npad * elem_bytes(ctx->storage);
    if (bytes != raw + 8) return fail(ctx, LBM_ERR_ARG, "wrong state size");
    int64_t phase = 0;
    memcpy(&phase, static_cast<const char *>(host) + raw, 8);
    if (phase != 0 && (phase != 1 || ctx->streaming != LBM_STREAM_AA))
        return fail(ctx, LBM_ERR_ARG, "state blob phase does not match the context's streaming");
    CK(ctx, cudaMemcpyAsync(ctx->f_cur, host, raw, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx, cudaMemsetAsync(ctx->err_flag, 0, 4, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->aa_swapped = phase == 1;
    ctx->state_undefined = false;
    return LBM_OK;
}

HGB_API lbm_status lbm_get_links(lbm_ctx *ctx, int32_t *nbr, uint8_t *link) {
    if (!ctx || ((!nbr || !link) && ctx->n)) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    const int q = ctx->q;
    const int64_t n = ctx->n, npad = ctx->npad;
    if (n == 0) return LBM_OK;
    std::vector<int32_t> tab((size_t)(q - 1) * npad);
    CK(ctx, cudaMemcpyAsync(tab.data(), ctx->tab, tab.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    const std::vector<int32_t> &perm = ctx->perm_host;
    for (int64_t xi = 0; xi < n; ++xi) {
        const int64_t x = perm[(size_t)xi];
        nbr[x] = (int32_t)x;
        link[x] = 0;
        for (int j = 1; j < q; ++j) {
            const int32_t s = tab[(size_t)(opp(j) - 1) * npad + xi];
            nbr[(int64_t)j * n + x] = s >= 0 ? perm[(size_t)s] : -1;
            link[(int64_t)j * n + x] = (uint8_t)(s >= 0 ? 0 : is_bfl(s) ? 1 : -s);
        }
    }
    return LBM_OK;
}

// ------------------------------------------------------------- adjoint

namespace {

// beta(s, r) = C(s + r, s): the number of steps that s checkpoints (the
// start state included) can reverse when each step is advanced at most r
// times (Griewank, "Achieving logarithmic growth of temporal and spatial
// complexity in reverse automatic differentiation", 1992).  Saturates.
int64_t binom_beta(int64_t s, int64_t r) {
    if (s < 0 || r < 0) return 0;
    const int64_t k = std::min(s, r), n = s + r;
    const int64_t cap = int64_t(1) << 62;
    int64_t v = 1;
    for (int64_t i = 1; i <= k; ++i) {
        // v = C(n - k + i, i), exact at every step
        const __int128 w = (__int128)v * (n - k + i) / i;
        if (w > cap) return cap;
        v = (int64_t)w;
    }
    return v;
}

// smallest r with beta(f + 1, r) >= l (f free slots plus the start state)
int64_t revolve_reps(int64_t l, int64_t f) {
    int64_t r = 0;
    while (binom_beta(f + 1, r) < l) ++r;
    return r;
}

// First checkpoint position for reversing l >= 2 steps with f >= 1 free
// slots: the smallest m with m <= beta(s, r-1) (the left part, already
// advanced once, is reversed with r-1 more advances) and l - m <= beta(s-1, r)
// (the right part with one slot less), raised to beta(s, r-2) so that the
// left part needs all its r-1 advances; s = f + 1.  With this split the
// total number of forward steps equals r l - beta(f + 2, r - 1), the minimum.
int64_t revolve_split(int64_t l, int64_t f) {
    const int64_t s = f + 1, r = revolve_reps(l, f);
    int64_t m = std::max<int64_t>({1, l - binom_beta(s - 1, r), binom_beta(s, r - 2)});
    return std::min<int64_t>(m, l - 1);
}

int64_t revolve_steps(int64_t l, int64_t f) {
    if (l <= 1) return 0;
    if (f == 0) return l * (l - 1) / 2;
    const int64_t m = revolve_split(l, f);
    return m + revolve_steps(l - m, f - 1) + revolve_steps(m, f);
}

struct AdjointRun {
    lbm_ctx *c;
    std::vector<void *> slots;
    std::vector<int> free_slots;
    void *W[2] = {nullptr, nullptr};
    float *lam[2] = {nullptr, nullptr};
    int lc = 0;
    double *acc_block = nullptr, *io_acc = nullptr;
    const double *weight = nullptr;
    int kind = 0;
    double scale = 1.0;
    int64_t t_begin = 0, t_end = 0, t0 = 0, T = 0;
    void *final_buf = nullptr;  // receives f(T)
    bool terminal_done = false;
    int64_t fwd_steps = 0, adj_steps = 0;
    // AA form: states in the AA layouts (the state of time t swapped when
    // p0 + t - t0 is odd), recomputation in place after an out-of-place first
    // step, one adjoint buffer lam[0] updated in place by the AA adjoint
    bool aa = false, p0 = false;
    bool swapped_at(int64_t t) const { return (((p0 ? 1 : 0) + (t - t0)) & 1) != 0; }

    AdjObjective objective_at(int64_t t) const {
        AdjObjective o{};
        o.active = (t >= t_begin && t < t_end) ? 1 : 0;
        o.kind = kind;
        o.scale = scale;
        o.weight = weight;
        const double tau = (double)c->L.tau;
        o.inv_tau2 = 1.0 / (tau * tau);
        o.wss_dlog = (0.5 / (tau * tau)) / (1.0 - 0.5 / tau);
        o.inv_tau2_f = (float)o.inv_tau2;
        o.wss_dlog_f = (float)o.wss_dlog;
        o.scale_f = (float)scale;
        return o;
    }
    AdjStep adj_step(int64_t t) const {
        AdjStep a{};
        a.io = iolet_step(c, t);
        for (int k = 0; k < c->n_iolets; ++k) {
            if (c->io_period[k] != 0.0) {
                const double arg = 2.0 * M_PI * (double)t / c->io_period[k] + c->io_phase[k];
                a.dsin[k] = std::sin(arg);
                a.dacos[k] = c->io_amp[k] != 0.0 ? c->io_amp[k] * std::cos(arg) : 0.0;
            }
        }
        return a;
    }
    cudaError_t step(const void *in, void *out, int64_t t) {
        ++fwd_steps;
        if (aa) {
            const bool odd = swapped_at(t);
            if (in == out) return launch_step_aa(c->L, out, odd, iolet_step(c, t), nullptr, c->stream, side());
            return launch_step_aa_oop(c->L, in, out, odd, iolet_step(c, t), c->stream);
        }
        return launch_step(c->L, in, out, iolet_step(c, t), nullptr, c->stream, side());
    }
    // m steps from the state src of time a; the result lands in dst
    cudaError_t advance(const void *src, int64_t a, int64_t m, void *dst) {
        if (aa) {
            for (int64_t k = 0; k < m; ++k) {
                cudaError_t e = step(k == 0 ? src : dst, dst, a + k);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        }
        const void *in = src;
        const bool dst_is_work = dst == W[0] || dst == W[1];
        void *other = dst == W[0] ? W[1] : W[0];
        for (int64_t k = 0; k < m; ++k) {
            void *out;
            if (k == m - 1) out = dst;
            else if (dst_is_work) out = ((m - 1 - k) % 2 == 0) ? dst : other;
            else out = W[k & 1];
            cudaError_t e = step(in, out, a + k);
            if (e != cudaSuccess) return e;
            in = out;
        }
        return cudaSuccess;
    }
    // the side stream of the context (null: none): the launch of the sites
    // with iolet links runs beside the bulk launch, as in lbm_step
    const SideStream *side() const { return c->side.s ? &c->side : nullptr; }
    cudaError_t adjoint(const void *state, const float *next, float *out, int64_t t) {
        const SideStream *sd = side();
        cudaStream_t io_stream = c->stream;
        if (sd) {
            cudaError_t e = cudaEventRecord(sd->fork, c->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(sd->s, sd->fork, 0);
            if (e != cudaSuccess) return e;
            io_stream = sd->s;
        }
        cudaError_t e =
            aa ? launch_adjoint_aa(c->L, state, swapped_at(t), out, next != nullptr, adj_step(t), objective_at(t),
                                   acc_block, io_acc, c->stream, io_stream)
               : launch_adjoint(c->L, state, next, out, adj_step(t), objective_at(t), acc_block, io_acc,
                                c->stream, io_stream);
        if (sd) {
            // join even after a failed launch, so that nothing is left forked
            const cudaError_t e2 = cudaEventRecord(sd->join, sd->s);
            const cudaError_t e3 = e2 == cudaSuccess ? cudaStreamWaitEvent(c->stream, sd->join, 0) : e2;
            if (e == cudaSuccess) e = e3;
        }
        return e;
    }
    // adjoint of step k (state of time k in `state`); the first call also
    // forms f(T) in the context's buffer and the terminal adjoint lam(T)
    cudaError_t adjoint_at(int64_t k, const void *state) {
        cudaError_t e;
        if (!terminal_done) {
            if ((e = step(state, final_buf, T - 1)) != cudaSuccess) return e;
            if ((e = adjoint(final_buf, nullptr, lam[lc], T)) != cudaSuccess) return e;
            terminal_done = true;
        }
        if (aa) {
            if ((e = adjoint(state, lam[0], lam[0], k)) != cudaSuccess) return e;  // in place
        } else {
            if ((e = adjoint(state, lam[lc], lam[1 - lc], k)) != cudaSuccess) return e;
            lc = 1 - lc;
        }
        ++adj_steps;
        return cudaSuccess;
    }
    // reverse the steps a .. b-1, the state of time a being in sa, with f free slots
    cudaError_t reverse(int64_t a, int64_t b, void *sa, int64_t f) {
        cudaError_t e;
        if (b - a == 1) return adjoint_at(a, sa);
        if (f == 0) {
            for (int64_t k = b - 1; k > a; --k) {
                if ((e = advance(sa, a, k - a, W[0])) != cudaSuccess) return e;
                if ((e = adjoint_at(k, W[0])) != cudaSuccess) return e;
            }
            return adjoint_at(a, sa);
        }
        const int64_t m = revolve_split(b - a, f);
        const int slot = free_slots.back();
        free_slots.pop_back();
        void *sm = slots[(size_t)slot];
        if ((e = advance(sa, a, m, sm)) != cudaSuccess) return e;
        if ((e = reverse(a + m, b, sm, f - 1)) != cudaSuccess) return e;
        free_slots.push_back(slot);
        return reverse(a, a + m, sa, f);
    }
};

}  // namespace

HGB_API lbm_status lbm_revolve_steps(int64_t nsteps, int32_t n_snap, int64_t *forward_steps) {
    if (nsteps < 0 || n_snap < 1 || !forward_steps)
        return fail(nullptr, LBM_ERR_ARG, "need nsteps >= 0, n_snap >= 1, forward_steps");
    *forward_steps = nsteps == 0 ? 0 : revolve_steps(nsteps, n_snap - 1) + 1;
    return LBM_OK;
}

HGB_API lbm_status lbm_set_tau(lbm_ctx *ctx, double tau) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(ctx, LBM_ERR_ARG, "tau must be finite and > 0.5");
    ctx->tau = tau;
    ctx->L.omega = (float)(1.0 / tau);
    ctx->L.tau = (float)tau;
    graphs_reset(ctx);  // the captured launches hold the old value
    return LBM_OK;
}

HGB_API lbm_status lbm_set_iolets(lbm_ctx *ctx, int32_t n_iolets, const double *rho_mean,
                                  const double *amp, const double *period, const double *phase) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (n_iolets != ctx->n_iolets) return fail(ctx, LBM_ERR_ARG, "n_iolets differs from the context's");
    lbm_params p{};
    p.q = ctx->q;
    p.storage = ctx->storage;
    p.tau = ctx->tau;
    p.rho0 = ctx->rho0;
    p.fp16_scale_log2 = ctx->scale_log2;
    p.n_iolets = n_iolets;
    p.rho_mean = rho_mean;
    p.amp = amp;
    p.period = period;
    p.phase = phase;
    p.iolet_kind = ctx->io_kind;
    p.iolet_normal = &ctx->io_normal[0][0];
    lbm_status st = validate_params(&p);
    if (st != LBM_OK) return fail(ctx, st, g_err);
    for (int k = 0; k < n_iolets; ++k) {
        ctx->io_mean[k] = rho_mean[k];
        ctx->io_amp[k] = amp[k];
        ctx->io_period[k] = period[k];
        ctx->io_phase[k] = phase[k];
    }
    return LBM_OK;
}

HGB_API lbm_status lbm_objective_grad(lbm_ctx *ctx, const lbm_objective *obj, int64_t nsteps,
                                      int32_t n_snap, double *J, double *dJ_dtau, double *dJ_dmean,
                                      double *dJ_damp, double *dJ_dphase, double *dJ_df0) {
    const Range range("lbm_objective_grad");
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!obj || (obj->kind != LBM_OBJ_WSS && obj->kind != LBM_OBJ_DENSITY))
        return fail(ctx, LBM_ERR_ARG, "objective kind must be LBM_OBJ_WSS or LBM_OBJ_DENSITY");
    if (ctx->n > 0 && !obj->weight) return fail(ctx, LBM_ERR_ARG, "objective weight is NULL");
    if (!std::isfinite(obj->scale)) return fail(ctx, LBM_ERR_ARG, "objective scale is not finite");
    if (nsteps < 0 || n_snap < 1) return fail(ctx, LBM_ERR_ARG, "need nsteps >= 0 and n_snap >= 1");
    if (!J) return fail(ctx, LBM_ERR_ARG, "J is NULL");
    if (ctx->state_undefined)
        return fail(ctx, LBM_ERR_STATE, "the state is undefined after a failed step; replace it with "
                    "lbm_set_state or lbm_set_populations");
    const int q = ctx->q, K = ctx->n_iolets;
    const int64_t n = ctx->n, npad = ctx->npad;
    const size_t sbytes = (size_t)q * npad * elem_bytes(ctx->storage);
    const int64_t nblk = std::max(1, adjoint_blocks(ctx->L));
    const int64_t nio = n - ctx->L.n_bulk;
    const size_t need_all = (size_t)(n_snap + 1) * sbytes + 2 * (size_t)q * npad * 4 + (size_t)npad * 8 +
                            (size_t)nblk * 16 + 3 * (size_t)std::max<int64_t>(nio, 1) * (q - 1) * 8 +
                            (size_t)(2 + 3 * LBM_MAX_IOLETS) * 8 + (dJ_df0 ? (size_t)q * n * 8 : 0);
    const size_t need = need_all > ctx->ws.bytes ? need_all - ctx->ws.bytes : 0;
    size_t free_b = 0, total_b = 0;
    CK(ctx, cudaMemGetInfo(&free_b, &total_b));
    if (need > 0 && need + (64u << 20) > free_b) {
        char msg[200];
        snprintf(msg, sizeof msg, "adjoint needs %zu bytes of device memory (%d snapshots), %zu free",
                 need, n_snap, free_b);
        return fail(ctx, LBM_ERR_NOMEM, msg);
    }
    AdjointRun R;
    R.c = ctx;
    R.kind = obj->kind == LBM_OBJ_WSS ? 0 : 1;
    R.scale = obj->scale;
    R.t_begin = obj->t_begin;
    R.t_end = obj->t_end;
    R.t0 = ctx->t;
    R.T = ctx->t + nsteps;
    cudaError_t e = cudaSuccess;
    auto &ws = ctx->ws;
    auto grow = [&](void **p, size_t b) {
        if (e != cudaSuccess || *p) return;
        e = cudaMalloc(p, b ? b : 16);
        if (e == cudaSuccess) {
            ws.bytes += b;
            ctx->device_bytes += b;
        }
    };
    // the per-context sizes of everything but the snapshots never change
    const bool aa = ctx->streaming == LBM_STREAM_AA;
    grow(&ws.W1, sbytes);
    if (aa) grow(&ws.W0, sbytes);
    grow((void **)&ws.lam[0], (size_t)q * npad * 4);
    grow((void **)&ws.lam[1], (size_t)q * npad * 4);
    grow((void **)&ws.weight, (size_t)npad * 8);
    grow((void **)&ws.acc_block, (size_t)nblk * 16);
    grow((void **)&ws.io_acc, 3 * (size_t)std::max<int64_t>(nio, 1) * (q - 1) * 8);
    grow((void **)&ws.out, (size_t)(2 + 3 * LBM_MAX_IOLETS) * 8);
    if (dJ_df0) grow((void **)&ws.lam0, (size_t)q * std::max<int64_t>(n, 1) * 8);
    while (e == cudaSuccess && ws.slots.size() < (size_t)n_snap) {
        void *p = nullptr;
        e = cudaMalloc(&p, sbytes);
        if (e == cudaSuccess) {
            ws.slots.push_back(p);
            ws.bytes += sbytes;
            ctx->device_bytes += sbytes;
        }
    }
    for (auto &ev : ws.ev)
        if (e == cudaSuccess && !ev) e = cudaEventCreate(&ev);
    if (e != cudaSuccess) {
        free_workspace(ctx);
        return cuda_fail(ctx, e, "lbm_objective_grad workspace");
    }
    R.slots.assign(ws.slots.begin(), ws.slots.begin() + n_snap);
    R.W[1] = ws.W1;
    R.W[0] = aa ? ws.W0 : ctx->f_nxt;
    R.final_buf = ctx->f_cur;  // f(t0) is copied into slot 0 first
    R.aa = aa;
    R.p0 = aa && ctx->aa_swapped;
    R.lam[0] = ws.lam[0];
    R.lam[1] = ws.lam[1];
    R.acc_block = ws.acc_block;
    R.io_acc = ws.io_acc;
    double *weight_dev = ws.weight, *out_dev = ws.out, *lam0_dev = ws.lam0;
    std::vector<double> wint((size_t)npad, 0.0);
    for (int64_t xi = 0; xi < n; ++xi) wint[(size_t)xi] = obj->weight[ctx->perm_host[(size_t)xi]];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(weight_dev, wint.data(), wint.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(R.acc_block, 0, (size_t)nblk * 16, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(R.io_acc, 0, 3 * (size_t)std::max<int64_t>(nio, 1) * (q - 1) * 8, ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(out_dev, 0, (size_t)(2 + 3 * K) * 8, ctx->stream);
    R.weight = weight_dev;
    for (int i = n_snap - 1; i >= 1; --i) R.free_slots.push_back(i);
    if (e == cudaSuccess) e = cudaEventRecord(ws.ev[0], ctx->stream);
    // slot 0 receives f(t0) in the context's own layout (pull, or the AA
    // layout of the context's phase)
    if (e == cudaSuccess) e = cudaMemcpyAsync(R.slots[0], ctx->f_cur, sbytes, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) {
        if (nsteps == 0) {
            e = R.adjoint(R.slots[0], nullptr, R.lam[0], R.t0);
            R.lc = 0;
            if (e == cudaSuccess && !aa)
                e = cudaMemcpyAsync(ctx->f_cur, R.slots[0], sbytes, cudaMemcpyDeviceToDevice, ctx->stream);
        } else {
            e = R.reverse(R.t0, R.T, R.slots[0], n_snap - 1);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(ws.ev[1], ctx->stream);
    if (e == cudaSuccess) e = launch_adjoint_final(ctx->L, R.acc_block, R.io_acc, out_dev, ctx->stream);
    if (e == cudaSuccess && dJ_df0) {
        const float *lam0 = R.lam[R.lc];
        if (aa && R.p0) {
            // lam(t0) of an AA context in the swapped phase is in swapped form
            DevLattice Lf = ctx->L;
            Lf.storage = 0;
            e = launch_relayout(Lf, R.lam[0], LAYOUT_AA_SWAPPED, R.lam[1], LAYOUT_NATURAL, ctx->stream);
            lam0 = R.lam[1];
        }
        if (e == cudaSuccess) e = launch_lam_to_caller(ctx->L, lam0, lam0_dev, ctx->stream);
    }
    std::vector<double> out((size_t)(2 + 3 * K), 0.0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out.data(), out_dev, out.size() * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && dJ_df0 && n > 0)
        e = cudaMemcpyAsync(dJ_df0, lam0_dev, (size_t)q * n * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    float sweep_ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&sweep_ms, ws.ev[0], ws.ev[1]);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "lbm_objective_grad");
    ctx->last_sweep_ms = sweep_ms;
    ctx->t = R.T;
    if (aa) ctx->aa_swapped = R.swapped_at(R.T);
    ctx->last_fwd_steps = R.fwd_steps;
    ctx->last_adj_steps = R.adj_steps;
    double jsum = out[0];
    if (obj->kind == LBM_OBJ_DENSITY) {
        // the kernel sums m (rho - rho0); add rho0 sum(m) for every state of
        // the window that the run visits (t0 .. t0 + nsteps)
        double msum = 0.0;
        for (int64_t x = 0; x < n; ++x) msum += obj->weight[x];
        const int64_t lo = std::max<int64_t>(R.t0, obj->t_begin);
        const int64_t hi = std::min<int64_t>(R.T, obj->t_end - 1);
        if (hi >= lo) jsum += (double)(hi - lo + 1) * (double)ctx->L.rho0 * msum;
    }
    *J = obj->scale * jsum;
    if (dJ_dtau) *dJ_dtau = out[1];
    for (int k = 0; k < K; ++k) {
        if (dJ_dmean) dJ_dmean[k] = out[(size_t)(2 + k)];
        if (dJ_damp) dJ_damp[k] = out[(size_t)(2 + K + k)];
        if (dJ_dphase) dJ_dphase[k] = out[(size_t)(2 + 2 * K + k)];
    }
    if (!std::isfinite(*J)) return fail(ctx, LBM_ERR_UNSTABLE, "non-finite objective");
    return LBM_OK;
}

HGB_API lbm_status lbm_adjoint_counts(const lbm_ctx *ctx, int64_t *forward_steps, int64_t *adjoint_steps,
                                      double *sweep_ms) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (forward_steps) *forward_steps = ctx->last_fwd_steps;
    if (adjoint_steps) *adjoint_steps = ctx->last_adj_steps;
    if (sweep_ms) *sweep_ms = ctx->last_sweep_ms;
    return LBM_OK;
}

HGB_API lbm_status lbm_release_workspace(lbm_ctx *ctx) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    free_workspace(ctx);
    return LBM_OK;
}

HGB_API lbm_status lbm_info(const lbm_ctx *ctx, int64_t *n, int64_t *npad, size_t *device_bytes) {
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (n) *n = ctx->n;
    if (npad) *npad = ctx->npad;
    if (device_bytes) *device_bytes = ctx->device_bytes;
    return LBM_OK;
}

HGB_API lbm_status lbm_slab_chunks(const lbm_ctx *ctx, int32_t *count) {
    if (!ctx || !count) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    *count = ctx->slab_chunks.empty() ? 0 : (int32_t)ctx->slab_chunks.size() - 1;
    return LBM_OK;
}

// ------------------------------------------------------------------ rendering

namespace {

void free_volume(lbm_volume *v) {
    if (!v) return;
    if (v->tex_lin) cudaDestroyTextureObject(v->tex_lin);
    if (v->tex_pt) cudaDestroyTextureObject(v->tex_pt);
    if (v->surf) cudaDestroySurfaceObject(v->surf);
    if (v->arr) cudaFreeArray(v->arr);
    cudaFree(v->occ);
    cudaFree(v->dist);
    delete v;
}

cudaMemcpy3DParms linear_copy(lbm_volume *v, float *lin, bool to_array) {
    cudaMemcpy3DParms cp{};
    cudaPitchedPtr pp = make_cudaPitchedPtr(lin, (size_t)v->dims[0] * 4, (size_t)v->dims[0],
                                            (size_t)v->dims[1]);
    if (to_array) {
        cp.srcPtr = pp;
        cp.dstArray = v->arr;
    } else {
        cp.srcArray = v->arr;
        cp.dstPtr = pp;
    }
    cp.extent = make_cudaExtent((size_t)v->dims[0], (size_t)v->dims[1], (size_t)v->dims[2]);
    cp.kind = cudaMemcpyDeviceToDevice;
    return cp;
}

bool finite3(const double *a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

}  // namespace

HGB_API lbm_status lbm_volume_create(int32_t nx, int32_t ny, int32_t nz, lbm_volume **out) {
    if (!out) return fail(nullptr, LBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || nx > 16384 || ny > 16384 || nz > 16384)
        return fail(nullptr, LBM_ERR_ARG, "volume dimensions must lie in [1, 16384]");
    lbm_volume *v = new lbm_volume();
    v->dims[0] = nx;
    v->dims[1] = ny;
    v->dims[2] = nz;
    for (int a = 0; a < 3; ++a) v->bdims[a] = (v->dims[a] + 7) / 8;
    v->occ_bytes = (size_t)v->bdims[0] * v->bdims[1] * v->bdims[2];
    const size_t need = (size_t)nx * ny * nz * 4 + 2 * v->occ_bytes;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e == cudaSuccess && need + (64u << 20) > free_b) {
        free_volume(v);
        return fail(nullptr, LBM_ERR_NOMEM, "the volume does not fit in device memory");
    }
    cudaChannelFormatDesc ch = cudaCreateChannelDesc<float>();
    if (e == cudaSuccess)
        e = cudaMalloc3DArray(&v->arr, &ch, make_cudaExtent((size_t)nx, (size_t)ny, (size_t)nz),
                              cudaArraySurfaceLoadStore);
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->occ, v->occ_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void **)&v->dist, v->occ_bytes);
    if (e == cudaSuccess) {
        cudaResourceDesc rd{};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = v->arr;
        cudaTextureDesc td{};
        for (int a = 0; a < 3; ++a) td.addressMode[a] = cudaAddressModeClamp;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        td.filterMode = cudaFilterModeLinear;
        e = cudaCreateTextureObject(&v->tex_lin, &rd, &td, nullptr);
        td.filterMode = cudaFilterModePoint;
        if (e == cudaSuccess) e = cudaCreateTextureObject(&v->tex_pt, &rd, &td, nullptr);
        if (e == cudaSuccess) e = cudaCreateSurfaceObject(&v->surf, &rd);
    }
    // a fresh volume holds zeros and no occupied brick
    if (e == cudaSuccess) e = launch_volume_clear(v->surf, v->dims, nullptr);
    if (e == cudaSuccess) e = cudaMemset(v->occ, 0, v->occ_bytes);
    if (e == cudaSuccess) e = launch_brick_distance(v->occ, v->dist, v->bdims, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_volume(v);
        return cuda_fail(nullptr, e, "lbm_volume_create");
    }
    *out = v;
    return LBM_OK;
}

HGB_API void lbm_volume_destroy(lbm_volume *vol) {
    if (!vol) return;
    cudaDeviceSynchronize();
    free_volume(vol);
}

HGB_API lbm_status lbm_volume_upload(lbm_volume *vol, const float *v_d, void *cuda_stream) {
    if (!vol || !v_d) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    const cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaMemcpy3DParms cp = linear_copy(vol, const_cast<float *>(v_d), true);
    CK(nullptr, cudaMemcpy3DAsync(&cp, s));
    CK(nullptr, cudaMemsetAsync(vol->occ, 0, vol->occ_bytes, s));
    CK(nullptr, launch_occupancy(v_d, vol->dims, vol->occ, vol->bdims, s));
    CK(nullptr, launch_brick_distance(vol->occ, vol->dist, vol->bdims, s));
    vol->lattice_serial = 0;
    return LBM_OK;
}

HGB_API lbm_status lbm_volume_download(const lbm_volume *vol, float *v_d, void *cuda_stream) {
    if (!vol || !v_d) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    cudaMemcpy3DParms cp = linear_copy(const_cast<lbm_volume *>(vol), v_d, false);
    CK(nullptr, cudaMemcpy3DAsync(&cp, (cudaStream_t)cuda_stream));
    return LBM_OK;
}

HGB_API lbm_status lbm_lattice_box(const lbm_ctx *ctx, int32_t *lo, int32_t *dims) {
    if (!ctx || !lo || !dims) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a) {
        lo[a] = ctx->box_lo[a];
        dims[a] = ctx->box_dims[a];
    }
    return LBM_OK;
}

HGB_API lbm_status lbm_volume_from_lattice(lbm_volume *vol, lbm_ctx *ctx, int32_t quantity,
                                           const int32_t *origin) {
    const Range range("lbm_volume_from_lattice");
    if (!ctx) return fail(nullptr, LBM_ERR_ARG, "ctx is NULL");
    if (!vol || !origin) return fail(ctx, LBM_ERR_ARG, "NULL argument");
    if (quantity < LBM_QTY_DENSITY || quantity > LBM_QTY_WSS)
        return fail(ctx, LBM_ERR_ARG, "unknown quantity");
    if (ctx->n == 0) return LBM_OK;
    if (!ctx->vox) {
        CK(ctx, cudaMalloc((void **)&ctx->vox, (size_t)ctx->n * 8));
        CK(ctx, cudaMemcpy(ctx->vox, ctx->vox_host.data(), (size_t)ctx->n * 8, cudaMemcpyHostToDevice));
    }
    VolumeTarget V{};
    V.surf = vol->surf;
    for (int a = 0; a < 3; ++a) {
        V.dims[a] = vol->dims[a];
        V.bdims[a] = vol->bdims[a];
        const int64_t sh = (int64_t)ctx->box_lo[a] - origin[a];
        if (sh < -(1LL << 30) || sh > (1LL << 30)) return fail(ctx, LBM_ERR_ARG, "origin out of range");
        V.shift[a] = (int)sh;
    }
    V.quantity = quantity;
    V.occ = vol->occ;
    const bool same = vol->lattice_serial == ctx->serial && vol->shift[0] == V.shift[0] &&
                      vol->shift[1] == V.shift[1] && vol->shift[2] == V.shift[2];
    if (!same) {
        // voxels without a site hold 0; bricks are flagged from the site positions
        CK(ctx, launch_volume_clear(vol->surf, vol->dims, ctx->stream));
        CK(ctx, cudaMemsetAsync(vol->occ, 0, vol->occ_bytes, ctx->stream));
    }
    V.mark = same ? 0 : 1;
    CK(ctx, launch_volume_fill(ctx->L, ctx->f_cur, cur_layout(ctx), ctx->vox, V, ctx->stream));
    if (!same) CK(ctx, launch_brick_distance(vol->occ, vol->dist, vol->bdims, ctx->stream));
    vol->lattice_serial = ctx->serial;
    for (int a = 0; a < 3; ++a) vol->shift[a] = V.shift[a];
    return LBM_OK;
}

HGB_API lbm_status lbm_render(const lbm_volume *vol, const lbm_view *view, float *rgba_d,
                              void *cuda_stream) {
    const Range range("lbm_render");
    if (!vol || !view || !rgba_d) return fail(nullptr, LBM_ERR_ARG, "NULL argument");
    if (((uintptr_t)rgba_d & 15) != 0) return fail(nullptr, LBM_ERR_ARG, "rgba_d must be 16-byte aligned");
    const lbm_view &w = *view;
    if (w.width < 1 || w.height < 1 || w.width > 16384 || w.height > 16384)
        return fail(nullptr, LBM_ERR_ARG, "image size must lie in [1, 16384]");
    if (!finite3(w.eye) || !finite3(w.center) || !finite3(w.up))
        return fail(nullptr, LBM_ERR_ARG, "eye, center and up must be finite");
    if (!(w.fov_y > 0.0 && w.fov_y < 3.1)) return fail(nullptr, LBM_ERR_ARG, "fov_y must lie in (0, 3.1)");
    if (!std::isfinite(w.tf_scale) || !std::isfinite(w.tf_offset))
        return fail(nullptr, LBM_ERR_ARG, "tf_scale and tf_offset must be finite");
    if (!(w.a_stop > 0.0 && w.a_stop <= 1.0)) return fail(nullptr, LBM_ERR_ARG, "a_stop must lie in (0, 1]");
    if (w.filter != LBM_FILTER_TEXTURE && w.filter != LBM_FILTER_EXACT)
        return fail(nullptr, LBM_ERR_ARG, "unknown filter");
    if (w.skip_empty != 0 && w.skip_empty != 1) return fail(nullptr, LBM_ERR_ARG, "skip_empty must be 0 or 1");
    const double diag = std::sqrt((double)vol->dims[0] * vol->dims[0] + (double)vol->dims[1] * vol->dims[1] +
                                  (double)vol->dims[2] * vol->dims[2]);
    if (!(w.dt >= 1e-3) || !(diag / w.dt <= (double)(1 << 24)))
        return fail(nullptr, LBM_ERR_ARG, "dt must be >= 1e-3 and leave at most 2^24 segments per ray");
    for (int e = 0; e < 256; ++e)
        for (int c = 0; c < 4; ++c)
            if (!std::isfinite(w.lut[e][c])) return fail(nullptr, LBM_ERR_ARG, "LUT entries must be finite");
    // camera basis in float64: forward, right = forward x up, up' = right x forward
    double f[3], r[3], u[3];
    for (int a = 0; a < 3; ++a) f[a] = w.center[a] - w.eye[a];
    const double fn = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    if (!(fn > 0.0)) return fail(nullptr, LBM_ERR_ARG, "eye and center coincide");
    for (double &x : f) x /= fn;
    r[0] = f[1] * w.up[2] - f[2] * w.up[1];
    r[1] = f[2] * w.up[0] - f[0] * w.up[2];
    r[2] = f[0] * w.up[1] - f[1] * w.up[0];
    const double un = std::sqrt(w.up[0] * w.up[0] + w.up[1] * w.up[1] + w.up[2] * w.up[2]);
    const double rn = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (!(rn > 1e-9 * un)) return fail(nullptr, LBM_ERR_ARG, "up is parallel to the view direction");
    for (double &x : r) x /= rn;
    u[0] = r[1] * f[2] - r[2] * f[1];
    u[1] = r[2] * f[0] - r[0] * f[2];
    u[2] = r[0] * f[1] - r[1] * f[0];
    RenderArgs a{};
    for (int c = 0; c < 3; ++c) {
        a.eye[c] = (float)w.eye[c];
        a.fwd[c] = (float)f[c];
        a.right[c] = (float)r[c];
        a.up[c] = (float)u[c];
        a.dims[c] = vol->dims[c];
        a.bdims[c] = vol->bdims[c];
    }
    const double th = std::tan(0.5 * w.fov_y);
    a.sx_mul = (float)(th * w.width / w.height);
    a.sy_mul = (float)th;
    a.dt = (float)w.dt;
    a.tf_scale = (float)w.tf_scale;
    a.tf_offset = (float)w.tf_offset;
    a.a_stop = (float)w.a_stop;
    a.width = w.width;
    a.height = w.height;
    a.filter = w.filter;
    std::memcpy(a.lut, w.lut, sizeof a.lut);
    // Skipping is exact when a sample of value 0 gets zero opacity: the
    // kernel's float arithmetic for v = 0, repeated here, must select LUT
    // entries whose alpha is 0 (both of them when it interpolates).
    bool zero_alpha_at_zero;
    {
        const float s0 = std::min(std::max((0.0f - a.tf_offset) * a.tf_scale, 0.0f), 1.0f) * 255.0f;
        const int l0 = std::min((int)s0, 254);
        const float fl = s0 - (float)l0;
        zero_alpha_at_zero = w.lut[l0][3] == 0.0f && (fl == 0.0f || w.lut[l0 + 1][3] == 0.0f);
    }
    a.skip = (w.skip_empty && zero_alpha_at_zero) ? 1 : 0;
    if (w.counters_d && ((uintptr_t)w.counters_d & 7) != 0)
        return fail(nullptr, LBM_ERR_ARG, "counters_d must be 8-byte aligned");
    a.counters = w.counters_d;
    CK(nullptr, launch_render(a, vol->tex_lin, vol->tex_pt, vol->dist, rgba_d, (cudaStream_t)cuda_stream));
    return LBM_OK;
}
