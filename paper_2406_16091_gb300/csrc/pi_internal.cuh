// pi_internal.cuh -- definitions shared by the libpi translation units.
//
// A context holds S >= 1 independent systems (pi_create makes S = 1).  Their
// particles, cells and X-rows are concatenated in system order, so one
// launch of each kernel covers every system; per-system geometry lives in a
// device array of SysDesc, and the first particle / cell / X-row of each
// system in three base arrays (S + 1 entries each).
//
// Layout of the device state (one cudaMalloc arena):
//   Ctrl            control words (scan ticket, error bits, M_C, row counters)
//   counts[C]       particles per cell (C = cells of all systems)
//   xbins[C]        per cell, where its XSUB x-sub-bins start (k_stabilise)
//   pbase[S+1]      first particle of each system in the current step
//   offsets[C+1]    exclusive scan of counts; offsets[C] = n
//   scan_status[T]  decoupled-lookback tile descriptors (T = scan tiles)
//   sys[S], cbase[S+1], wbase[S+1], kscale[2S]  per-system constants
//   cell[n_max]     cell of each input particle            (binning scratch)
//   rank[n_max]     provisional slot inside its cell        (binning scratch)
//   rec[n_max]      32-byte Rec per particle in unstable slot order (binning
//                   scratch): one full DRAM sector per random write
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
    ERR_CHECK = 8u,  // a bounds check of the debug build failed (PI_CHECK)
};

struct Ctrl {
    uint32_t ticket;        // next scan tile to hand out
    uint32_t error;         // ERR_* bits, sticky until the next pi_bin
    uint32_t max_per_cell;  // M_C of the last pi_bin (over all systems)
    uint32_t n;             // particle count of the last pi_bin
    uint32_t work[2];       // next work item handed out by the tiled interaction;
                            // launch number q uses work[q & 1] and clears the other
    uint32_t check_site;    // debug builds: the first failed bounds check (CheckSite)
    uint32_t pad0;
    unsigned long long ovf; // bucketed binning: overflow buckets, count << 40 | their particles
    unsigned long long evals; // direct kernels: target-source evaluations (PI_OPT_COUNT_EVALS)
    uint32_t tickets[3];    // scan tile tickets of a step's second to fourth scans (radix binning)
    uint32_t pad[49];       // the control block is 256 bytes
};

// Grid geometry.  inv_w[d] = fl32(n[d] / (hi[d] - lo[d])) computed in FP64.
struct Grid {
    float lo[3];
    float hi[3];
    float inv_w[3];
    int32_t n[3];
};

// One system's constants.
struct SysDesc {
    Grid g;
    float cell_w[3];  // (hi - lo) / n, computed in FP64
    float rc2;        // fl32(r_c * r_c)
    float slack;      // absolute margin of the conservative x-windows
    uint32_t cell_base;
    uint32_t work_base;  // first work item of the tiled interaction
    uint32_t nseg;       // work items per X-row: segments of SEG_CELLS cells
    uint32_t row_base;   // first X-row (rows are counted over all systems)
};

// P holds the sorted particles with ROW_PADS sentinel slots after every
// X-row: sorted index k of X-row r (global) is P index k + ROW_PADS * r.
// Loops that read four sources at a time may then run up to three slots
// past a window's end without leaving the row's particles and sentinels.
constexpr int ROW_PADS = 3;

// The tiled interaction's work items are segments of SEG_CELLS consecutive
// cells of an X-row; rows longer than that are split so that heavy rows do
// not leave one CTA working alone at the end.
constexpr int SEG_CELLS = 32;

constexpr int MAX_SYSTEMS = 2048;

// Threads per block of the direct interaction kernels (the host deals out
// their blocks when a launch covers a list of P ranges).
constexpr int DIRECT_BLOCK = 128;

// The systems as kernels see them.
struct Systems {
    const SysDesc* sys;     // [S]
    const uint32_t* pbase;  // [S+1] first particle (= first sorted slot) of each system
    const uint32_t* cbase;  // [S+1] first cell
    const uint32_t* wbase;  // [S+1] first work item of the tiled interaction
    const uint32_t* rbase;  // [S+1] first X-row
    int S;
};

// Largest s with base[s] <= v (base[0] = 0, nondecreasing).
__device__ __forceinline__ int find_system(const uint32_t* base, int S, uint32_t v)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Scan tiling (a3): 256 threads x 16 counts per tile.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// x-sub-bins per cell.  A particle of cell cx lies in sub-bin
// clamp(floor((x - lo) * XSUB * inv_w) - XSUB * cx, 0, XSUB - 1), which is
// monotone in x along an X-row; k_stabilise stores where each sub-bin of a
// cell starts, and the tiled interaction uses them to find x-windows.
constexpr int XSUB = 8;

// Flags in the top byte of a cell's sub-bin word (xbins[c].y >> 24):
// XBIN_COARSE, more than 255 members (the byte counts would overflow, so
// every sub-bin starts at the cell); XBIN_DENSE, more than DENSE_CELL
// members (the sub-bin starts are valid, but an interaction may prefer
// exact window bounds from a binary search of the x-sorted members).
constexpr uint32_t XBIN_COARSE = 1u, XBIN_DENSE = 2u;
constexpr uint32_t DENSE_CELL = 255;

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

// Bounds checks of the debug build (compiled with -DPI_CHECK).  Each
// checked access names its site; an index outside its array sets ERR_CHECK
// in the error word, records the first failing site in Ctrl::check_site,
// and the access is skipped instead of made, so a bad index shows up as a
// status (PI_ERR_CHECK from pi_sync_status) rather than a fault.  Normal
// builds compile every check to `true`.
enum CheckSite : uint32_t {
    CS_HIST_COUNTS = 1,      // k_hist: counts[cell]
    CS_SCATTER_REC = 2,      // k_scatter: rec[slot]
    CS_STAB_MEMBER = 3,      // k_stabilise: rec[q] of a cell's members
    CS_STAB_OUT = 4,         // k_stabilise: perm / sx / sy / sz / P / xbins
    CS_DIRECT_SRC = 5,       // direct interaction: four-source trip from P
    CS_DIRECT_WIN = 6,       // direct interaction: window list in shared memory
    CS_DIRECT_LOOKUP = 7,    // direct interaction: offsets / xbins of a window bound
    CS_DIRECT_TARGET = 8,    // direct interaction: target slots and outputs
    CS_STAGED_BUF = 9,       // staged interaction: staged rows, pads, source reads
    CS_STAGED_TABLE = 10,    // staged interaction: sub-bin lookup table
    CS_PPNL_SRC = 11,        // Alg. 1: sorted sources of the stencil
    CS_SCAN_TILE = 12,       // k_scan: tile descriptors
};

#ifdef PI_CHECK
__device__ __forceinline__ bool pi_in_bounds(Ctrl* ctrl, uint64_t i, uint64_t n, uint32_t site)
{
    if (i < n) return true;
    atomicOr(&ctrl->error, ERR_CHECK);
    atomicCAS(&ctrl->check_site, 0u, site);
    return false;
}
#define PI_BOUNDS(ctrl, i, n, site) ::pi::pi_in_bounds((ctrl), (uint64_t)(i), (uint64_t)(n), (site))
#else
#define PI_BOUNDS(ctrl, i, n, site) true
#endif

// x-sub-bin of a particle at x in cell c_local of grid g: clamp(floor((x -
// lo) * XSUB * inv_w) - XSUB * cx, 0, XSUB - 1), monotone in x along an
// X-row (FP32, the same rounding everywhere it is computed).
__device__ __forceinline__ int x_sub_bin(float x, uint32_t c_local, const Grid& g)
{
    const float invs = g.inv_w[0] * (float)XSUB;
    const int cxs = XSUB * (int)(c_local % (uint32_t)g.n[0]);
    return min(max(__float2int_rd(__fmul_rn(__fsub_rn(x, g.lo[0]), invs)) - cxs, 0), XSUB - 1);
}

// The thermometer of sub-bin sb: byte b - 1 is 1 when sb < b (b = 1 ..
// XSUB - 1), as (bytes 0..3, bytes 4..6); summed over a cell's members it
// gives how many of them lie below each sub-bin boundary.
__device__ __forceinline__ uint2 thermometer(int sb)
{
    static_assert(XSUB == 8, "the thermometer has 7 one-byte counts");
    const unsigned long long t = 0x01010101010101ull & (~0ull << (8 * sb));
    return make_uint2((uint32_t)t, (uint32_t)(t >> 32));
}

// The system of input particle i (its particle base is the largest <= i).
__device__ __forceinline__ int system_of_particle(const Systems& sy, uint32_t i)
{
    return sy.S == 1 ? 0 : find_system(sy.pbase, sy.S, i);
}

// Four consecutive input particles i0 .. i0 + 3 below `end`, as float4 loads
// when the arrays are 16-byte aligned and the group is whole.
__device__ __forceinline__ void load4(const float* x, const float* y, const float* z, uint32_t i0, uint32_t end,
                                      int vec, float (&px)[4], float (&py)[4], float (&pz)[4], bool (&valid)[4])
{
    if (vec && i0 + 4u <= end) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(x + i0));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(y + i0));
        const float4 c = __ldcs(reinterpret_cast<const float4*>(z + i0));
        px[0] = a.x; px[1] = a.y; px[2] = a.z; px[3] = a.w;
        py[0] = b.x; py[1] = b.y; py[2] = b.z; py[3] = b.w;
        pz[0] = c.x; pz[1] = c.y; pz[2] = c.z; pz[3] = c.w;
#pragma unroll
        for (int j = 0; j < 4; ++j) valid[j] = true;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            valid[j] = i0 + j < end;
            px[j] = valid[j] ? x[i0 + j] : 0.f;
            py[j] = valid[j] ? y[i0 + j] : 0.f;
            pz[j] = valid[j] ? z[i0 + j] : 0.f;
        }
    }
}

// Global cells of four consecutive particles (the systems advance along
// the group as in k_hist); `ok` collects the out-of-box test.
__device__ __forceinline__ void cells4(const Systems& sy, uint32_t i0, const float (&px)[4], const float (&py)[4],
                                       const float (&pz)[4], const bool (&valid)[4], uint32_t (&cell)[4], bool& ok)
{
    int s = system_of_particle(sy, i0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (sy.S > 1 && valid[j])
            while (s + 1 < sy.S && i0 + j >= __ldg(sy.pbase + s + 1)) ++s;
        const SysDesc& d = sy.sys[s];
        bool in = true;
        cell[j] = cell_of(px[j], py[j], pz[j], d.g, in) + d.cell_base;
        ok &= in | !valid[j];
    }
}

__device__ __forceinline__ uint32_t load_error(const Ctrl* ctrl)
{
    return *((volatile const uint32_t*)&ctrl->error);
}

// The control block's error word and M_C as the kernels before this one left
// them, read by one thread of the CTA and shared through shared memory: when
// every thread reads the one line itself, the requests queue at the single
// L2 slice that holds it.  Every thread of the CTA must call it (it holds a
// barrier), once per kernel.
__device__ __forceinline__ uint2 cta_ctrl_words(const Ctrl* ctrl)
{
    __shared__ uint2 s_words;
    if (threadIdx.x == 0) s_words = make_uint2(load_error(ctrl), *((volatile const uint32_t*)&ctrl->max_per_cell));
    __syncthreads();
    return s_words;
}

__device__ __forceinline__ uint32_t cta_error(const Ctrl* ctrl) { return cta_ctrl_words(ctrl).x; }

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch.  A kernel started by launch_dependent may
// begin while the kernel before it in the stream is still running (once
// every block of that kernel has called pdl_trigger or exited); pdl_wait
// then blocks until that kernel has completed and its writes are visible.
// Whatever a kernel reads or writes of the step's state comes after its
// pdl_wait.  For a kernel launched the ordinary way both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_dependent(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// One particle in provisional (unstable) slot order: position, input index,
// cell, and its x-sub-bin as a thermometer (byte b - 1 is 1 when the
// sub-bin is < b, b = 1 .. XSUB - 1; t_lo holds bytes 0..3, t_hi bytes
// 4..6), so that summing the thermometers of a cell's members gives the
// cell's sub-bin starts.  32 bytes, aligned, so that the scatter writes
// whole DRAM sectors; (x, i, t_lo, t_hi) come first: what the ranking reads
// of every member.
struct __align__(32) Rec {
    float x;
    uint32_t i;
    uint32_t t_lo, t_hi;
    float y, z;
    uint32_t c;
    uint32_t pad;
};
static_assert(sizeof(Rec) == 32, "one DRAM sector per record");

// Parameters of k_zero: clear [p, p + n_words), then write the S + 1
// particle bases of this step.
template <int NB>
struct ZeroArgs {
    uint32_t* p;
    size_t n_words;
    uint32_t* pbase;
    int nb;  // entries of vals used (S + 1)
    uint32_t vals[NB];
};

static_assert(sizeof(Ctrl) == 256, "the control block is 256 bytes");

// Bucketed binning (pi_bucket.cu).  The cells are split into B buckets of
// 2^bc_log2 consecutive cells and the particles into chunks of `chunk`
// consecutive input particles.  mat[b * chunks + k] counts the particles of
// chunk k in bucket b; its exclusive scan (k_scan) in that bucket-major
// order gives where chunk k's particles of bucket b start in bucket order,
// and where every bucket starts.  One CTA per bucket then ranks the
// bucket's cells in shared memory; buckets of more than BUCKET_CAP
// particles go through a grid-wide path instead.
constexpr int BUCKET_CAP = 2048;           // particles of a bucket ranked in shared memory
constexpr int BUCKET_MAX_CELLS = 1024;     // cells per bucket
constexpr int BUCKET_MAX = 8192;           // buckets (the chunk kernels' shared histogram)
constexpr int BUCKET_CHUNK = 8192;         // particles per chunk
struct BucketPlan {
    uint32_t bc_log2;  // cells per bucket = 1 << bc_log2
    uint32_t B;        // buckets
    uint32_t chunks;   // chunks of BUCKET_CHUNK particles
    uint32_t C;        // cells of all systems
};
// Radix binning (pi_radix.cu): a least-significant-digit radix sort of the
// particles by global cell, digits of at most RADIX_MAX_BITS bits over
// chunks of RADIX_CHUNK particles; the digit x chunk count matrices live in
// the bucketed path's `mat` buffers.
constexpr int RADIX_CHUNK = 4096;
constexpr int RADIX_MAX_BITS = 9;
struct RadixPlan {
    uint32_t passes;      // digit passes, at most 4 (cells < 2^31)
    uint32_t digit_bits;  // bits per digit
    uint32_t bins;        // 1 << digit_bits
    uint32_t chunks;
    uint32_t C;
};
bool radix_plan(uint64_t n, uint64_t C, uint64_t mat_capacity, RadixPlan& plan);
cudaError_t launch_radix_keys(const float* x, const float* y, const float* z, uint32_t n, const Systems& sy,
                              const RadixPlan& plan, uint32_t* keys, uint32_t* mat, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_radix_count(const uint32_t* keys, uint32_t n, const RadixPlan& plan, uint32_t shift,
                               uint32_t* mat, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_radix_scatter(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                 uint32_t* vals_out, uint32_t n, const RadixPlan& plan, uint32_t shift,
                                 const uint32_t* base, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_radix_gather(const uint32_t* keys, const uint32_t* vals, const float* x, const float* y,
                                const float* z, uint32_t n, uint32_t C, uint32_t* offsets, uint32_t* perm, float* sx,
                                float* sy_out, float* sz, Ctrl* ctrl, int num_sms, cudaStream_t s);
cudaError_t launch_radix_rank(const uint32_t* keys, uint32_t n, const Systems& sy, uint32_t C,
                              const uint32_t* offsets, const uint32_t* perm, const float* sx, const float* sy_in,
                              const float* sz, uint32_t* counts, float4* P, uint2* xbins, Ctrl* ctrl, int num_sms,
                              cudaStream_t s);

// Whether the bucketed path takes n particles in C cells, and its plan.
bool bucket_plan(uint64_t n, uint64_t C, uint64_t mat_capacity, BucketPlan& plan);
cudaError_t launch_bucket_count(const float* x, const float* y, const float* z, uint32_t n, const Systems& sy,
                                const BucketPlan& plan, uint32_t* mat, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_bucket_scatter(const float* x, const float* y, const float* z, uint32_t n,
                                  const Systems& sy, const BucketPlan& plan, const uint32_t* base, float4* rec,
                                  Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_bucket_cells(const float4* rec, uint32_t n, const Systems& sy, const BucketPlan& plan,
                                const uint32_t* base, uint32_t* counts, uint32_t* offsets, uint32_t* perm,
                                float* sx, float* sy_out, float* sz, float4* P, uint2* xbins, float4* rec2,
                                uint2* ovf_list, Ctrl* ctrl, cudaStream_t s);
cudaError_t launch_bucket_big(const float4* rec2, uint32_t n, const Systems& sy, const BucketPlan& plan,
                              const uint32_t* offsets, uint32_t* perm, float* sx, float* sy_out, float* sz,
                              float4* P, uint2* xbins, const uint2* ovf_list, Ctrl* ctrl, int num_sms,
                              cudaStream_t s);

// Launch wrappers (each returns the cudaGetLastError of its launch).
cudaError_t launch_zero(uint32_t* p, size_t n_words, uint32_t* pbase, const uint32_t* vals, int nb,
                        cudaStream_t s);
cudaError_t launch_hist(const float* x, const float* y, const float* z, uint32_t n,
                        const Systems& sy, uint32_t* counts, uint32_t* cell, uint32_t* rank,
                        Ctrl* ctrl, int num_sms, cudaStream_t s);
// track_max: also record the largest count in Ctrl::max_per_cell (M_C);
// ticket_slot: 0 takes the tiles from Ctrl::ticket, 1..3 from
// Ctrl::tickets[slot - 1] (each scan of a step needs its own, cleared by
// k_zero, and its own epoch)
cudaError_t launch_scan(const uint32_t* counts, uint32_t C, uint32_t* offsets,
                        unsigned long long* status, Ctrl* ctrl, uint32_t epoch,
                        uint64_t wait_limit_ns, int withhold_first, cudaStream_t s, int track_max = 1,
                        int ticket_slot = 0);
cudaError_t launch_scatter(const uint32_t* cell, const uint32_t* rank, const float* x,
                           const float* y, const float* z, uint32_t n, const Systems& sy,
                           const uint32_t* offsets, Rec* rec, Ctrl* ctrl, int num_sms, cudaStream_t s);
cudaError_t launch_stabilise(const Rec* rec, uint32_t n,
                             const Systems& sy, const uint32_t* offsets, uint32_t* perm, float* sx,
                             float* sy_out, float* sz, float4* P, uint2* xbins, Ctrl* ctrl,
                             int num_sms, cudaStream_t s);

// FP64 total of v over the particles of each system (out[S], device), in a
// fixed order: `parts` partial sums per system in `partial` [S * parts].
constexpr int TOTAL_PARTS = 32;
cudaError_t launch_total_f64(const float* v, const Systems& sy, double* partial, int parts,
                             double* out, cudaStream_t s);

// Writes one system's constants (system 0 of a context) from launch
// parameters: sys[0] = d, cbase[1] = cells, wbase[1] = work items.
cudaError_t launch_set_system(SysDesc* sys, uint32_t* cbase, uint32_t* wbase, uint32_t* rbase,
                              const SysDesc& d, uint32_t cells, uint32_t work, uint32_t rows, cudaStream_t s);

// Copies count words from host memory into device memory by kernel
// launches whose parameters carry them (no host-side staging, so the copy
// may be captured in a CUDA graph); vals is read before the call returns.
cudaError_t launch_write_words(uint32_t* dst, const uint32_t* vals, size_t count, cudaStream_t s);

// Per-system scales of the interaction kernel, written from launch
// parameters (vals[i] for i < count, count <= 2 MAX_SYSTEMS) into kscale.
cudaError_t launch_set_kscale(float* kscale, const float* vals, int count, cudaStream_t s);

// Interaction kernels (PI_KERNEL_* of include/pi.h), and the Gaussian with
// a compensated exponent that the host picks for short kernel lengths
// (r_c^2 / h^2 > FINE_GAUSS_RATIO), where the plain FP32 exponent's rounding
// would exceed the accuracy the sums are held to.
enum : int { KERNEL_GAUSSIAN = 0, KERNEL_LJ = 1, KERNEL_LOWFLOP = 2, KERNEL_HIGHFLOP = 3, KERNEL_GAUSSIAN_FINE = 4 };
constexpr double FINE_GAUSS_RATIO = 16.0;

struct InteractArgs {
    Systems sy;
    const float4* P;        // x-ordered copy: (x, y, z, stable slot as bits)
    const uint2* xbins;     // per cell: starts of its XSUB x-sub-bins (see k_stabilise)
    const float* sx;
    const float* sy_pos;
    const float* sz;
    const uint32_t* offsets;
    const uint32_t* perm;
    uint32_t n;             // particles of all systems
    uint32_t np;            // entries of P: n plus ROW_PADS per X-row
    uint32_t work;          // work items (X-row segments) of all systems
    const float* kscale;    // [2S]: scale t of system s at [s] (Gaussian K = 2^(r2 t), t =
                            // -log2(e)/h^2 in FP32; Lennard-Jones sigma^2), the FP32
                            // remainder of the FP64 scale at [S + s] (fine Gaussian)
    float kscale0;          // the scale and remainder when S == 1 (kscale may then be null)
    float kscale0_lo;
    int kernel;             // KERNEL_*
    float one, zero;        // 1 and 0, opaque to the compiler (high-FLOP kernel)
    float* S;
    float* Vx;
    float* Vy;
    float* Vz;
    uint32_t* nbr;
    int original_order;
    Ctrl* ctrl;
    uint64_t wait_limit_ns; // bound of every device-side wait
    uint32_t seq;           // launch number of the tiled kernel (row counter slot)
    // direct kernels only: a launch over some systems of a batch covers the
    // P ranges [ranges[r].x, ranges[r].y), r < nranges, range r starting at
    // block rblock[r] (range_blocks blocks in all); null: all of P
    const uint2* ranges;
    const uint32_t* rblock;
    int nranges;
    unsigned range_blocks;
    int count_evals;        // direct kernels: add their evaluations to ctrl->evals
};

// Each adds the number of kernels it launched to *launches.
cudaError_t launch_interact_ppnl(const InteractArgs& a, bool kahan, int num_sms, cudaStream_t s,
                                 int* launches);
// tile: 0, 1, 2 = one CTA per chunk with 32, 64, 128 threads (two targets
// each); 3, 4 = warp-specialised, 4 or 8 consumer warps; 5 = direct (no
// staging, sources through L1, two targets per thread); 6 = direct with
// four targets per thread; per_sm[tile] = resident CTAs.
constexpr int NUM_TILES = 7;
constexpr int DEFAULT_TILE = 5;         // PI_TILE_AUTO below 8 particles per cell, or not the packed sums
constexpr int HIGH_OCCUPANCY_TILE = 6;  // PI_TILE_AUTO: plain Gaussian / low-FLOP sums from 8 per cell
cudaError_t launch_interact_tiled(const InteractArgs& a, bool kahan, int num_sms, const int* per_sm,
                                  int tile, cudaStream_t s, int* launches);
// Resident CTAs per SM of each tile shape of the tiled kernel (per_sm[NUM_TILES]).
cudaError_t tiled_occupancy(bool kahan, int* per_sm);

}  // namespace pi
