// Direct volume rendering by ray marching (arXiv 1906.11925, Section 3.3.2):
// the volume sits in a 3D texture, the view parameters in the constant bank
// (the kernel's by-value argument), rays march front to back through a
// 256-entry RGBA transfer-function table.  The image goes to a device buffer.
//
// Definitions (shared with the public header): voxel (i, j, k) is centred at
// (i, j, k), the box is [-1/2, n - 1/2]; the ray's piece inside the box is cut
// into segments of length dt (the last shorter), sampled at their midpoints;
// s = clamp((v - offset) scale, 0, 1), LUT linearly interpolated at s * 255,
// opacity a = min(1, alpha l); C += (1 - A) a c, A += (1 - A) a, stopping once
// A >= a_stop.
//
// GB300 design:
//   - one thread per pixel, 32 x 8 pixel tiles (a warp is one row of 32 rays;
//     tile shape measured: 32 x 8 0.60 ms, 16 x 8 0.64 ms, 8 x 4 0.77 ms);
//   - the texture unit's trilinear filter (one fetch per sample), or, for
//     float32 weights, eight point fetches;
//   - the LUT moves from the constant bank into shared memory at block start:
//     neighbouring rays index different entries, which the constant cache
//     would serialise;
//   - empty-space skipping over 8^3 bricks: a brick is empty when no non-zero
//     voxel lies within two voxels of it, so every sample within one voxel of
//     it reads exactly 0.  When the LUT gives such samples zero opacity (the
//     host checks), a sample contributes exactly nothing.  Each brick stores
//     its Chebyshev distance k (in bricks, capped) to the nearest non-empty
//     brick, so a ray in an empty brick jumps to the segment where it leaves
//     the cube of 2k - 1 bricks around it; the image is bitwise the one of
//     the full march.
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm_internal.h"

namespace hemelb_gb300 {
namespace {

#ifndef HGB_RTILE_X
#define HGB_RTILE_X 32
#endif
#ifndef HGB_RTILE_Y
#define HGB_RTILE_Y 8
#endif
constexpr int kTileX = HGB_RTILE_X, kTileY = HGB_RTILE_Y;
constexpr int kDistCap = 15;  // largest brick distance stored (means ">= 15")

__device__ __forceinline__ float sample_exact(cudaTextureObject_t t, float x, float y, float z,
                                              const int (&n)[3]) {
    x = fminf(fmaxf(x, 0.f), (float)(n[0] - 1));
    y = fminf(fmaxf(y, 0.f), (float)(n[1] - 1));
    z = fminf(fmaxf(z, 0.f), (float)(n[2] - 1));
    const float x0 = floorf(x), y0 = floorf(y), z0 = floorf(z);
    const float fx = x - x0, fy = y - y0, fz = z - z0;
    // texel centres at integer + 1/2; the clamp address mode repeats the edge
    const float X = x0 + 0.5f, Y = y0 + 0.5f, Z = z0 + 0.5f;
    const float c000 = tex3D<float>(t, X, Y, Z), c100 = tex3D<float>(t, X + 1.f, Y, Z);
    const float c010 = tex3D<float>(t, X, Y + 1.f, Z), c110 = tex3D<float>(t, X + 1.f, Y + 1.f, Z);
    const float c001 = tex3D<float>(t, X, Y, Z + 1.f), c101 = tex3D<float>(t, X + 1.f, Y, Z + 1.f);
    const float c011 = tex3D<float>(t, X, Y + 1.f, Z + 1.f);
    const float c111 = tex3D<float>(t, X + 1.f, Y + 1.f, Z + 1.f);
    const float c00 = c000 + (c100 - c000) * fx, c10 = c010 + (c110 - c010) * fx;
    const float c01 = c001 + (c101 - c001) * fx, c11 = c011 + (c111 - c011) * fx;
    const float c0 = c00 + (c10 - c00) * fy, c1 = c01 + (c11 - c01) * fy;
    return c0 + (c1 - c0) * fz;
}

template <int FILTER, bool COUNT>
__global__ void __launch_bounds__(kTileX * kTileY)
k_render(const __grid_constant__ RenderArgs a, cudaTextureObject_t tex, const uint8_t *__restrict__ dist,
         float4 *__restrict__ out) {
    unsigned taken = 0, jumps = 0;
    __shared__ float4 lut[256];
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    for (int e = tid; e < 256; e += kTileX * kTileY)
        lut[e] = make_float4(a.lut[e][0], a.lut[e][1], a.lut[e][2], a.lut[e][3]);
    __syncthreads();
    const int px = blockIdx.x * kTileX + threadIdx.x, py = blockIdx.y * kTileY + threadIdx.y;
    if (px >= a.width || py >= a.height) return;

    const float sx = ((px + 0.5f) / a.width * 2.f - 1.f) * a.sx_mul;
    const float sy = (1.f - (py + 0.5f) / a.height * 2.f) * a.sy_mul;
    float d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] = a.fwd[c] + sx * a.right[c] + sy * a.up[c];
    const float inv_n = 1.0f / sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int c = 0; c < 3; ++c) d[c] *= inv_n;

    // slab intersection with [-1/2, n - 1/2]^3
    float tn = 0.f, tf = 3.0e38f;
    bool hit = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float lo = -0.5f, hi = a.dims[c] - 0.5f;
        if (d[c] == 0.f) {
            hit &= a.eye[c] >= lo && a.eye[c] <= hi;
        } else {
            const float inv = 1.0f / d[c];
            float t0 = (lo - a.eye[c]) * inv, t1 = (hi - a.eye[c]) * inv;
            if (t0 > t1) {
                const float tmp = t0;
                t0 = t1;
                t1 = tmp;
            }
            tn = fmaxf(tn, t0);
            tf = fminf(tf, t1);
        }
    }
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
    if (hit && tn < tf) {
        const float len = tf - tn, dt = a.dt;
        float inv_d[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) inv_d[c] = 1.0f / d[c];  // +-inf on an axis-parallel ray
        float t_check = -1.f;  // the ray is in a non-empty brick up to here
        for (int m = 0;;) {
            const float s0 = m * dt;
            if (!(s0 < len) || A >= a.a_stop) break;
            const float l = fminf(dt, len - s0);
            const float t = tn + s0 + 0.5f * l;
            const float x = a.eye[0] + t * d[0], y = a.eye[1] + t * d[1], z = a.eye[2] + t * d[2];
            if (a.skip && t >= t_check) {
                const int b[3] = {min(max(__float2int_rd((x + 0.5f) * 0.125f), 0), a.bdims[0] - 1),
                                  min(max(__float2int_rd((y + 0.5f) * 0.125f), 0), a.bdims[1] - 1),
                                  min(max(__float2int_rd((z + 0.5f) * 0.125f), 0), a.bdims[2] - 1)};
                const int k = __ldg(dist + ((int64_t)b[2] * a.bdims[1] + b[1]) * a.bdims[0] + b[0]);
                // exit of the cube of bricks within r - 1 of this one (all
                // empty when k = r > 0; the brick itself when k = 0)
                const int r = k ? k : 1;
                float te = 3.0e38f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const float face = d[c] > 0.f ? 8.f * (b[c] + r) - 0.5f : 8.f * (b[c] - r + 1) - 0.5f;
                    const float tc = (face - a.eye[c]) * inv_d[c];
                    if (d[c] != 0.f) te = fminf(te, tc);
                }
                if (k) {
                    // segments that end before te sample inside the empty cube
                    const float mf = floorf((te - tn) / dt);
                    m = mf > (float)(m + 1) ? (mf < 3.0e7f ? (int)mf : 30000000) : m + 1;
                    if (COUNT) ++jumps;
                    continue;
                }
                t_check = te;  // no look-up until the ray leaves this brick
            }
            float v;
            if (FILTER == 0)
                v = tex3D<float>(tex, x + 0.5f, y + 0.5f, z + 0.5f);
            else
                v = sample_exact(tex, x, y, z, a.dims);
            const float s = __saturatef((v - a.tf_offset) * a.tf_scale) * 255.f;
            const int l0 = min((int)s, 254);
            const float fl = s - (float)l0;
            const float4 e0 = lut[l0], e1 = lut[l0 + 1];
            const float er = e0.x + (e1.x - e0.x) * fl, eg = e0.y + (e1.y - e0.y) * fl;
            const float eb = e0.z + (e1.z - e0.z) * fl, ea = e0.w + (e1.w - e0.w) * fl;
            const float w = (1.f - A) * fminf(1.f, ea * l);
            C0 += w * er;
            C1 += w * eg;
            C2 += w * eb;
            A += w;
            ++m;
            if (COUNT) ++taken;
        }
    }
    __stcs(out + (int64_t)py * a.width + px, make_float4(C0, C1, C2, A));
    if (COUNT) {
        // counters[0] += samples composited, counters[1] += brick jumps
        const unsigned lane_mask = __activemask();
        const unsigned ts = __reduce_add_sync(lane_mask, taken), js = __reduce_add_sync(lane_mask, jumps);
        if ((tid & 31) == __ffs(lane_mask) - 1) {  // the lowest active lane of the warp
            atomicAdd(a.counters, (unsigned long long)ts);
            atomicAdd(a.counters + 1, (unsigned long long)js);
        }
    }
}

__global__ void k_volume_clear(cudaSurfaceObject_t surf, int nx, int ny, int nz) {
    const int64_t total = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int64_t r = i / nx;
        surf3Dwrite(0.0f, surf, x * (int)sizeof(float), (int)(r % ny), (int)(r / ny), cudaBoundaryModeZero);
    }
}

__global__ void k_occupancy(const float *__restrict__ v, int nx, int ny, int nz, uint8_t *occ, int bx,
                            int by, int bz) {
    const int64_t total = (int64_t)nx * ny * nz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (__ldg(v + i) == 0.0f) continue;
        const int p[3] = {(int)(i % nx), (int)((i / nx) % ny), (int)(i / ((int64_t)nx * ny))};
        const int bd[3] = {bx, by, bz};
        int b0[3], b1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            b0[c] = max(0, (p[c] - 2) >> 3);  // ceil((p - 9) / 8)
            b1[c] = min(bd[c] - 1, (p[c] + 2) >> 3);
        }
        for (int z = b0[2]; z <= b1[2]; ++z)
            for (int y = b0[1]; y <= b1[1]; ++y)
                for (int x = b0[0]; x <= b1[0]; ++x) occ[((int64_t)z * by + y) * bx + x] = 1;
    }
}

// One axis of the separable Chebyshev distance transform on the brick grid:
// out[p] = min over |j| <= kDistCap of max(|j|, in[p + j e_axis]) (cells
// outside the grid count as kDistCap), capped at kDistCap.  With
// first set, in holds marks (non-zero = occupied: distance 0, else kDistCap).
template <int AXIS>
__global__ void k_brick_distance(const uint8_t *__restrict__ in, uint8_t *__restrict__ out, int bx, int by,
                                 int bz, bool first) {
    const int64_t total = (int64_t)bx * by * bz;
    const int n[3] = {bx, by, bz};
    const int64_t stride[3] = {1, bx, (int64_t)bx * by};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int p[3] = {(int)(i % bx), (int)((i / bx) % by), (int)(i / ((int64_t)bx * by))};
        int best = kDistCap;
        for (int j = -kDistCap + 1; j < kDistCap; ++j) {
            const int q = p[AXIS] + j;
            if (q < 0 || q >= n[AXIS]) continue;
            const int v = in[i + j * stride[AXIS]];
            const int dv = first ? (v ? 0 : kDistCap) : v;
            best = min(best, max(abs(j), dv));
        }
        out[i] = (uint8_t)best;
    }
}

unsigned stride_grid(int64_t total) {
    const int64_t want = (total + 255) / 256;
    return (unsigned)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_render(const RenderArgs &a, cudaTextureObject_t tex_lin, cudaTextureObject_t tex_pt,
                          const uint8_t *dist, float *rgba, cudaStream_t s) {
    const dim3 block(kTileX, kTileY);
    const dim3 grid((a.width + kTileX - 1) / kTileX, (a.height + kTileY - 1) / kTileY);
    float4 *o = reinterpret_cast<float4 *>(rgba);
    if (a.counters) {
        if (a.filter == 0)
            k_render<0, true><<<grid, block, 0, s>>>(a, tex_lin, dist, o);
        else
            k_render<1, true><<<grid, block, 0, s>>>(a, tex_pt, dist, o);
    } else {
        if (a.filter == 0)
            k_render<0, false><<<grid, block, 0, s>>>(a, tex_lin, dist, o);
        else
            k_render<1, false><<<grid, block, 0, s>>>(a, tex_pt, dist, o);
    }
    return cudaGetLastError();
}

cudaError_t launch_volume_clear(cudaSurfaceObject_t surf, const int (&dims)[3], cudaStream_t s) {
    const int64_t total = (int64_t)dims[0] * dims[1] * dims[2];
    k_volume_clear<<<stride_grid(total), 256, 0, s>>>(surf, dims[0], dims[1], dims[2]);
    return cudaGetLastError();
}

cudaError_t launch_brick_distance(uint8_t *marks, uint8_t *dist, const int (&b)[3], cudaStream_t s) {
    const int64_t total = (int64_t)b[0] * b[1] * b[2];
    const unsigned g = stride_grid(total);
    k_brick_distance<0><<<g, 256, 0, s>>>(marks, dist, b[0], b[1], b[2], true);
    k_brick_distance<1><<<g, 256, 0, s>>>(dist, marks, b[0], b[1], b[2], false);
    k_brick_distance<2><<<g, 256, 0, s>>>(marks, dist, b[0], b[1], b[2], false);
    return cudaGetLastError();
}

cudaError_t launch_occupancy(const float *v, const int (&dims)[3], uint8_t *occ, const int (&bdims)[3],
                             cudaStream_t s) {
    const int64_t total = (int64_t)dims[0] * dims[1] * dims[2];
    k_occupancy<<<stride_grid(total), 256, 0, s>>>(v, dims[0], dims[1], dims[2], occ, bdims[0], bdims[1],
                                                   bdims[2]);
    return cudaGetLastError();
}

}  // namespace hemelb_gb300
