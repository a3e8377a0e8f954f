// pi_internal.cuh -- definitions shared by the libpi translation units.
//
// Layout of the device state of one context (one cudaMalloc arena):
//   Ctrl            control words (scan ticket, error bits, M_C)
//   counts[C]       particles per cell
//   xbins[C]        per cell, where its 4 x-sub-bins start in P (k_xorder)
//   offsets[C+1]    exclusive scan of counts; offsets[C] = n
//   scan_status[T]  decoupled-lookback tile descriptors (T = scan tiles)
//   cell[n_max]     cell of each input particle            (binning scratch)
//   rank[n_max]     provisional slot inside its cell        (binning scratch)
//   perm_u[n_max]   unstable slot -> input index            (binning scratch)
//   pos_u[n_max]    float4 (x, y, z, cell) in unstable slot order (binning scratch)
//   perm[n_max]     stable   slot -> input index
//   sx, sy, sz      positions in sorted order
//   P[n_max]        float4 (x, y, z, stable slot): sorted order, and inside
//                   each cell ordered by x -- what the tiled interaction stages
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pi {

// Device error bits (Ctrl::error).
enum : uint32_t {
    ERR_OUT_OF_BOX = 1u,
    ERR_TIMEOUT = 2u,
    ERR_CAPACITY = 4u,
};

struct Ctrl {
    uint32_t ticket;        // next scan tile to hand out
    uint32_t error;         // ERR_* bits, sticky until the next pi_bin
    uint32_t max_per_cell;  // M_C of the last pi_bin
    uint32_t n;             // particle count of the last pi_bin
    uint32_t work[2];       // next X-row handed out by the tiled interaction;
                            // launch number q uses work[q & 1] and clears the other
    uint32_t pad[58];       // the control block is 256 bytes
};

// Grid geometry.  inv_w[d] = fl32(n[d] / (hi[d] - lo[d])) computed in FP64.
struct Grid {
    float lo[3];
    float hi[3];
    float inv_w[3];
    int32_t n[3];
};

// Scan tiling (a3): 256 threads x 16 counts per tile.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Padding (in elements) after the sorted position arrays.
constexpr int SORTED_PAD = 16;

// Cell index of a position (Sec. 2: "compute its cell index using its
// physical position").  FP32, round-to-nearest subtract and multiply, floor,
// clamp; X fastest so that an X-row of cells is contiguous after sorting.
// `ok` is false when a coordinate is outside [lo, hi) or NaN; the returned
// cell is then still inside the grid.
__device__ __forceinline__ int axis_cell(float p, float lo, float inv_w, int n)
{
    float t = __fmul_rn(__fsub_rn(p, lo), inv_w);
    int c = __float2int_rd(t);  // floor; NaN -> 0, huge values saturate
    return min(max(c, 0), n - 1);
}

__device__ __forceinline__ uint32_t cell_of(float x, float y, float z, const Grid& g, bool& ok)
{
    ok = (x >= g.lo[0]) & (x < g.hi[0]) & (y >= g.lo[1]) & (y < g.hi[1]) & (z >= g.lo[2]) &
         (z < g.hi[2]);
    int cx = axis_cell(x, g.lo[0], g.inv_w[0], g.n[0]);
    int cy = axis_cell(y, g.lo[1], g.inv_w[1], g.n[1]);
    int cz = axis_cell(z, g.lo[2], g.inv_w[2], g.n[2]);
    return (uint32_t)cx + (uint32_t)g.n[0] * ((uint32_t)cy + (uint32_t)g.n[1] * (uint32_t)cz);
}

__device__ __forceinline__ uint32_t load_error(const Ctrl* ctrl)
{
    return *((volatile const uint32_t*)&ctrl->error);
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Launch wrappers (each returns the cudaGetLastError of its launch).
cudaError_t launch_zero(uint32_t* p, size_t n_words, cudaStream_t s);
cudaError_t launch_hist(const float* x, const float* y, const float* z, uint32_t n, const Grid& g,
                        uint32_t* counts, uint32_t* cell, uint32_t* rank, Ctrl* ctrl, int num_sms,
                        cudaStream_t s);
cudaError_t launch_scan(const uint32_t* counts, uint32_t C, uint32_t* offsets,
                        unsigned long long* status, Ctrl* ctrl, uint32_t epoch,
                        uint64_t wait_limit_ns, int withhold_first, cudaStream_t s);
cudaError_t launch_scatter(const uint32_t* cell, const uint32_t* rank, const float* x,
                           const float* y, const float* z, uint32_t n, const uint32_t* offsets,
                           uint32_t* perm_u, float4* pos_u, Ctrl* ctrl, int num_sms, cudaStream_t s);
cudaError_t launch_stabilise(const uint32_t* perm_u, const float4* pos_u, uint32_t n, const Grid& g,
                             const uint32_t* offsets, uint32_t* perm, float* sx, float* sy,
                             float* sz, float4* P, uint32_t* xbins, Ctrl* ctrl, int num_sms,
                             cudaStream_t s);

struct InteractArgs {
    const float4* P;        // x-ordered copy: (x, y, z, stable slot as bits)
    const uint32_t* xbins;  // per cell: starts of its 4 x-sub-bins (see k_xorder)
    const float* sx;
    const float* sy;
    const float* sz;
    const uint32_t* offsets;
    const uint32_t* perm;
    uint32_t n;
    Grid g;
    float rc2;     // fl32(r_c * r_c)
    float kscale;  // fl32(-log2(e) / h^2): K = 2^(r2 * kscale)
    float* S;
    float* Vx;
    float* Vy;
    float* Vz;
    uint32_t* nbr;
    int original_order;
    Ctrl* ctrl;
    float slack;            // absolute margin for the conservative windows
    uint64_t wait_limit_ns; // bound of every device-side wait
    uint32_t seq;           // launch number of the tiled kernel (row counter slot)
    float cell_w[3];        // cell widths (hi - lo) / n, computed in FP64
};

// Each adds the number of kernels it launched to *launches.
cudaError_t launch_interact_ppnl(const InteractArgs& a, bool kahan, int num_sms, cudaStream_t s,
                                 int* launches);
cudaError_t launch_interact_tiled(const InteractArgs& a, bool kahan, int num_sms,
                                  cudaStream_t s, int* launches);

}  // namespace pi
