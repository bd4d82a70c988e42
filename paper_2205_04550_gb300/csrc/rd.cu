// rd.cu -- the forward model of Section 2.1 (Eq. 1-2) on the GPU: the
// reaction-diffusion equation du/dt = div(D grad u) + rho u (1 - u) with a
// no-flux boundary, from a seed point, for a batch of parameter sets.
//
// Discretisation: unit voxel spacing, D(x) = D_w m(x) from a tissue map of
// relative diffusivities (domain = {m > 0}); the flux through the face of
// neighbours i, j is D_w h_ij (u_j - u_i) with h_ij the harmonic mean of
// m_i and m_j (zero when either is outside the domain: no flux through its
// boundary, Eq. 2; no flux through the grid's outer faces either); explicit
// Euler steps u <- u + a sum_j h_ij (u_j - u_i) + b u (1 - u) with a = dt D_w,
// b = dt rho, dt = T_end / n, n = ceil(T_end (6 D_w max m + rho) / cfl).
//
// Layout: u is [nz][ny][nx] binary32, two ping-pong buffers per simulation.
// The face coefficients of the map are computed once: hx[i] is the face
// between voxel i and its +x neighbour (0 on the last x column), hy and hz
// likewise, and hym[i] the face to the -y neighbour (0 on the first row);
// they are shared by every simulation of the batch (L2-resident at 128^3:
// 4 x 8 MiB).
//
// Simulations run in slots (continuous batching): a launch advances every
// busy slot by one step, and the host refills a slot whose simulation has
// ended with the next one between two launches.  A CTA owns a (32 VEC) x 8
// (x, y) tile of one slot -- VEC = 4 voxels per thread (float4 accesses)
// when nx is a multiple of 4, else 1 -- and streams it through an 8-voxel z
// range.  Two kinds of tile are skipped exactly:
//   * tiles without a domain voxel: their u is 0 at every step;
//   * tiles outside the box of L-infinity radius step+1 around the seed:
//     the 7-point stencil spreads the support by one voxel per step, so u
//     is still exactly 0 there (both buffers start zeroed and are never
//     written there).
#include "kernels.h"

namespace dbq {
namespace {

constexpr int kTileY = 8, kTileZ = 8;

// Voxels per thread along x: 4 (float4 loads) when rows are a multiple of 4
// voxels long, else 1.  A tile is 32 * VEC voxels wide.
__host__ __device__ constexpr int tile_x(int vec) { return 32 * vec; }
int vec_of(int nx) { return nx % 4 == 0 ? 4 : 1; }

__global__ void rd_faces_kernel(const float* __restrict__ m, int nx, int ny, int nz, int tx_w,
                                float* __restrict__ hx, float* __restrict__ hy,
                                float* __restrict__ hz, float* __restrict__ hym,
                                unsigned int* __restrict__ tile_any)
{
    const int64_t v = (int64_t)nx * ny * nz;
    const int tiles_x = (nx + tx_w - 1) / tx_w, tiles_y = (ny + kTileY - 1) / kTileY;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const int y = (int)((i / nx) % ny);
        const int z = (int)(i / ((int64_t)nx * ny));
        const float mi = m[i];
        const double a = mi;
        auto face = [a](float mj) -> float {
            const double b = mj;
            return (a + b > 0.0) ? (float)(2.0 * a * b / (a + b)) : 0.0f;
        };
        hx[i] = x + 1 < nx ? face(m[i + 1]) : 0.0f;
        hy[i] = y + 1 < ny ? face(m[i + nx]) : 0.0f;
        hz[i] = z + 1 < nz ? face(m[i + (int64_t)nx * ny]) : 0.0f;
        hym[i] = y > 0 ? face(m[i - nx]) : 0.0f;
        if (mi > 0.0f) {
            const int t = (x / tx_w) + tiles_x * ((y / kTileY) + tiles_y * (z / kTileZ));
            if (!tile_any[t]) tile_any[t] = 1u;
        }
    }
}

template <int VEC>
__device__ __forceinline__ void ldv(const float* p, float (&r)[VEC])
{
    if constexpr (VEC == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        r[0] = t.x;
        r[1] = t.y;
        r[2] = t.z;
        r[3] = t.w;
    } else {
        r[0] = *p;
    }
}

template <int VEC>
__device__ __forceinline__ void stv(float* p, const float (&r)[VEC])
{
    if constexpr (VEC == 4)
        *reinterpret_cast<float4*>(p) = make_float4(r[0], r[1], r[2], r[3]);
    else
        *p = r[0];
}

template <int VEC>
__device__ __forceinline__ void zero(float (&r)[VEC])
{
#pragma unroll
    for (int e = 0; e < VEC; ++e) r[e] = 0.0f;
}

// One step of every busy slot.  A warp owns one x-row of the tile, VEC
// consecutive voxels per lane: x-neighbours inside a lane are registers,
// across lanes shuffles, across the tile edge loads by the edge lanes; the
// y- and z-neighbours are loads (rows of the tile's other warps are L1
// hits).  No shared memory and no barriers; the loads of KZ planes are
// issued before their arithmetic.  Every load is unconditional: at a grid
// edge the missing neighbour's address is clamped to the voxel itself and
// its face coefficient is 0, and threads past the grid (or planes past the
// tile) read a clamped voxel and store nothing.  Offsets are 32-bit
// (V < 2^31).
template <int VEC>
__global__ void __launch_bounds__(256, 4)   // 64 registers: 32 warps per SM
rd_step_kernel(RdStepArgs g, int launch)
{
    constexpr int TX = tile_x(VEC);
    constexpr int KZ = VEC == 4 ? 2 : 4;
    const RdSim p = g.sims[blockIdx.z];
    const int step = launch - p.start;
    if (step < 0 || step >= p.steps) return;
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const int tiles_y = (ny + kTileY - 1) / kTileY;
    const int x0 = blockIdx.x * TX;
    const int y0 = (blockIdx.y % tiles_y) * kTileY;
    const int z0 = (blockIdx.y / tiles_y) * kTileZ;
    const int z1 = min(z0 + kTileZ, nz);
    if (!g.tile_any[blockIdx.x + gridDim.x * blockIdx.y]) return;
    const int r = step + 1;
    if (x0 + TX - 1 < p.sx - r || x0 > p.sx + r || y0 + kTileY - 1 < p.sy - r ||
        y0 > p.sy + r || z1 - 1 < p.sz - r || z0 > p.sz + r)
        return;
    const int plane = nx * ny;
    const int64_t v = (int64_t)plane * nz;
    if (threadIdx.x == 0 && threadIdx.y == 0 && g.updates)
        atomicAdd(g.updates, (unsigned long long)(min(TX, nx - x0) * min(kTileY, ny - y0) *
                                                  (z1 - z0)));
    const float* __restrict__ src = (step & 1 ? g.buf1 : g.buf0) + (int64_t)blockIdx.z * v;
    float* __restrict__ dst = (step & 1 ? g.buf0 : g.buf1) + (int64_t)blockIdx.z * v;
    const float* __restrict__ hx = g.hx;
    const float* __restrict__ hy = g.hy;
    const float* __restrict__ hz = g.hz;
    const float* __restrict__ hym = g.hym;
    const int lane = threadIdx.x;
    const int x = x0 + lane * VEC, y = y0 + threadIdx.y;
    const bool active = x < nx && y < ny;
    const int xc = min(x, nx - VEC), yc = min(y, ny - 1);
    const int col = xc + nx * yc;
    const int dym = yc > 0 ? nx : 0, dyp = yc + 1 < ny ? nx : 0;
    const bool edge_l = lane == 0 && xc > 0, edge_r = lane == 31 && xc + VEC < nx;
    float um[VEC], uc[VEC], hzm[VEC];
    ldv<VEC>(src + col + z0 * plane, uc);
    if (z0 > 0) {
        ldv<VEC>(src + col + (z0 - 1) * plane, um);
        ldv<VEC>(hz + col + (z0 - 1) * plane, hzm);
    } else {
        zero(um);
        zero(hzm);
    }
    const float a = p.a, b = p.b;
    for (int zb = z0; zb < z1; zb += KZ) {
        float up[KZ][VEC], ym[KZ][VEC], yp[KZ][VEC], cx[KZ][VEC], cy[KZ][VEC], cz[KZ][VEC],
            cym[KZ][VEC], exm[KZ], ecxm[KZ], exp_[KZ];
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int z = min(zb + k, z1 - 1);
            const int i = col + z * plane;
            const int dzp = z + 1 < nz ? plane : 0;
            ldv<VEC>(src + i + dzp, up[k]);
            ldv<VEC>(src + i - dym, ym[k]);
            ldv<VEC>(src + i + dyp, yp[k]);
            ldv<VEC>(hx + i, cx[k]);
            ldv<VEC>(hy + i, cy[k]);
            ldv<VEC>(hz + i, cz[k]);
            ldv<VEC>(hym + i, cym[k]);
            exm[k] = edge_l ? src[i - 1] : 0.0f;
            ecxm[k] = edge_l ? hx[i - 1] : 0.0f;
            exp_[k] = edge_r ? src[i + VEC] : 0.0f;
        }
#pragma unroll
        for (int k = 0; k < KZ; ++k) {
            const int z = zb + k;
            float left = __shfl_up_sync(0xffffffffu, uc[VEC - 1], 1);
            float right = __shfl_down_sync(0xffffffffu, uc[0], 1);
            float cleft = __shfl_up_sync(0xffffffffu, cx[k][VEC - 1], 1);
            if (lane == 0) {
                left = exm[k];
                cleft = ecxm[k];
            }
            if (lane == 31) right = exp_[k];
            float o[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const float u = uc[e];
                const float uxm = e ? uc[e > 0 ? e - 1 : 0] : left;
                const float cxm = e ? cx[k][e > 0 ? e - 1 : 0] : cleft;
                const float uxp = e < VEC - 1 ? uc[e < VEC - 1 ? e + 1 : 0] : right;
                float lap = cxm * (uxm - u);
                lap += cx[k][e] * (uxp - u);
                lap += cym[k][e] * (ym[k][e] - u);
                lap += cy[k][e] * (yp[k][e] - u);
                lap += hzm[e] * (um[e] - u);
                lap += cz[k][e] * (up[k][e] - u);
                o[e] = u + a * lap + b * u * (1.0f - u);
            }
            if (active && z < z1) stv<VEC>(dst + col + z * plane, o);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                um[e] = uc[e];
                uc[e] = up[k][e];
                hzm[e] = cz[k][e];
            }
        }
    }
}

}  // namespace

int rd_tiles(int nx, int ny, int nz)
{
    const int tw = tile_x(vec_of(nx));
    return ((nx + tw - 1) / tw) * ((ny + kTileY - 1) / kTileY) * ((nz + kTileZ - 1) / kTileZ);
}

cudaError_t launch_rd_faces(const float* m, int nx, int ny, int nz, float* hx, float* hy,
                            float* hz, float* hym, unsigned int* tile_any, cudaStream_t stream)
{
    cudaError_t err = cudaMemsetAsync(tile_any, 0, (size_t)rd_tiles(nx, ny, nz) * 4, stream);
    if (err != cudaSuccess) return err;
    const int64_t v = (int64_t)nx * ny * nz;
    const int64_t want = (v + 255) / 256;
    const int blocks = (int)(want < 152 * 16 ? want : 152 * 16);
    rd_faces_kernel<<<blocks, 256, 0, stream>>>(m, nx, ny, nz, tile_x(vec_of(nx)), hx, hy, hz,
                                                hym, tile_any);
    return cudaGetLastError();
}

cudaError_t launch_rd_step(const RdStepArgs& g, int slots, int launch, cudaStream_t stream)
{
    if (slots <= 0) return cudaSuccess;
    const int vec = vec_of(g.nx), tw = tile_x(vec);
    const dim3 grid((g.nx + tw - 1) / tw,
                    ((g.ny + kTileY - 1) / kTileY) * ((g.nz + kTileZ - 1) / kTileZ), slots);
    if (vec == 4)
        rd_step_kernel<4><<<grid, dim3(32, kTileY), 0, stream>>>(g, launch);
    else
        rd_step_kernel<1><<<grid, dim3(32, kTileY), 0, stream>>>(g, launch);
    return cudaGetLastError();
}

}  // namespace dbq
