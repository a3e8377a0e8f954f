// pi_api.cu -- host side of the libpi C ABI (declared in include/pi.h).
//
// Argument checks, the device arena of a context, the launch sequence of a
// step and the mapping of device error bits to pi_status.  No compute
// happens here: every step of the path is one of the kernels in pi_bin.cu
// and pi_interact.cu.  A context holds one or more independent systems; the
// single-system calls are the one-system case of the batch calls.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pi.h"
#include "pi_internal.cuh"

using pi::Ctrl;
using pi::Grid;
using pi::SysDesc;
using pi::Rec;

struct pi_ctx {
    int S;
    std::vector<pi_box> boxes;
    std::vector<float> rc;
    std::vector<int64_t> n_max;  // per system
    std::vector<SysDesc> sys;     // host copy of the per-system constants
    std::vector<uint32_t> cbase;  // [S+1]
    std::vector<uint32_t> wbase;  // [S+1]
    std::vector<uint32_t> rbase;  // [S+1] first X-row of each system
    int64_t C;                    // cells of all systems
    int64_t C_alloc;              // cells the arena was sized for
    int64_t rows = 0;             // X-rows of all systems
    int64_t n_max_total;
    uint32_t work;                // work items of the tiled interaction
    int device;
    int num_sms;
    int tiled_per_sm[2][pi::NUM_TILES];  // resident CTAs of each tile shape (plain, Kahan)

    // device arena and its parts
    void* arena;
    Ctrl* ctrl;
    uint32_t* counts;
    uint2* xbins;
    uint32_t* pbase;
    uint32_t* offsets;
    unsigned long long* scan_status;
    SysDesc* d_sys;
    uint32_t* d_cbase;
    uint32_t* d_wbase;
    uint32_t* d_rbase;
    float* d_kscale;
    double* d_partial;            // [S * TOTAL_PARTS] scratch of pi_total_f64
    uint32_t* cell;
    uint32_t* rank;
    Rec* rec;
    uint32_t* perm;
    float* sx;
    float* sy;
    float* sz;
    float4* P;

    // host-buffer path (allocated on first use)
    float* io;    // host-transfer staging: 3 input and 5 output arrays of io_n entries
    size_t io_n;

    int64_t n;                      // particles of the last pi_bin (all systems)
    std::vector<uint32_t> pbase_h;  // [S+1] particle bases of the last pi_bin
    std::vector<float> kscale_h;    // [2S] per-system kernel scales last written to d_kscale
    int binned;                     // a pi_bin has been enqueued since the last failure
    uint32_t epoch;                 // scan launch epoch
    uint64_t launches;              // kernels launched
    uint32_t tiled_seq;             // launches of the tiled interaction kernel
    int algo;
    int precision;
    int kernel;
    int tile;                       // tile shape of the tiled kernel (0 .. NUM_TILES - 1, or PI_TILE_AUTO)
    uint64_t wait_limit_ns;
    int withhold_scan;

    int binning;                    // PI_BIN_* (PI_OPT_BINNING)
    int count_evals;                // PI_OPT_COUNT_EVALS
    // bucketed binning: count matrix, its scan, overflow buckets
    uint32_t* mat;
    uint32_t* mat_base;
    uint2* ovf_list;
    size_t mat_cap;                 // entries of mat (mat_base has one more)

    // per-system tile shapes of a batch (empty: every system runs `tile`);
    // entries 5 or 6, or 0 for a system left out (autotuner trials only)
    std::vector<int> sys_tile;
    // device range lists of the per-system shapes: [0, 2S) the ranges of
    // shape 5, [2S, 4S) of shape 6, [4S, 5S) and [5S, 6S) their first blocks
    uint32_t* d_ranges;
    std::vector<uint32_t> ranges_h;  // what was last written there
};

namespace {

thread_local char g_last_error[512] = "";

pi_status cuda_fail(cudaError_t e, const char* what)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s)", what, cudaGetErrorName(e),
                  cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return PI_ERR_NOMEM;
    return PI_ERR_CUDA;
}

#define PI_TRY(call)                                       \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Makes the context's device current for the scope of a call.
struct DeviceScope {
    int prev = -1;
    bool changed = false;
    cudaError_t err = cudaSuccess;
    explicit DeviceScope(int dev)
    {
        err = cudaGetDevice(&prev);
        if (err == cudaSuccess && prev != dev) {
            err = cudaSetDevice(dev);
            changed = (err == cudaSuccess);
        }
    }
    ~DeviceScope()
    {
        if (changed) cudaSetDevice(prev);
    }
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Carves aligned pieces out of one allocation.
struct Carver {
    size_t off = 0;
    template <class T>
    size_t take(size_t count)
    {
        off = align_up(off, 256);
        size_t at = off;
        off += count * sizeof(T);
        return at;
    }
};

// Grid and margins of one system (Sec. 3: cell width >= r_c).
pi_status make_system(const pi_box& box, float r_c, SysDesc& d, int64_t& cells)
{
    if (!(r_c > 0.0f) || std::isinf(r_c)) return PI_ERR_INVALID_ARG;
    std::memset(&d, 0, sizeof d);
    cells = 1;
    float max_abs = 0.f, min_w = FLT_MAX;
    for (int k = 0; k < 3; ++k) {
        const double lo = box.lo[k], hi = box.hi[k];
        if (!std::isfinite(lo) || !std::isfinite(hi) || !(hi > lo)) return PI_ERR_INVALID_ARG;
        double n = std::floor((hi - lo) / (double)r_c);
        if (n < 1.0) n = 1.0;
        if (n > 2147483647.0) return PI_ERR_INVALID_ARG;
        d.g.lo[k] = box.lo[k];
        d.g.hi[k] = box.hi[k];
        d.g.n[k] = (int32_t)n;
        d.g.inv_w[k] = (float)(n / (hi - lo));
        d.cell_w[k] = (float)((hi - lo) / n);
        cells *= (int64_t)n;
        if (cells >= ((int64_t)1 << 31) - 1) return PI_ERR_INVALID_ARG;
        max_abs = std::fmax(max_abs, std::fmax(std::fabs(box.lo[k]), std::fabs(box.hi[k])));
        min_w = std::fmin(min_w, (float)((hi - lo) / n));
    }
    d.rc2 = r_c * r_c;  // FP32 product, round to nearest
    // margin of the conservative x-windows: cell assignment and face
    // positions are exact only up to a few ulp of the coordinates
    d.slack = 1e-5f * min_w + 16.0f * FLT_EPSILON * max_abs;
    return PI_OK;
}

// Scale t of the interaction kernel for length h (FP32).
float kernel_scale(int kernel, float h)
{
    const double hd = (double)h;
    switch (kernel) {
        case PI_KERNEL_LJ:
        case PI_KERNEL_HIGHFLOP: return h * h;  // sigma^2 in FP32
        case PI_KERNEL_LOWFLOP: return 0.f;
        default: return (float)(-1.4426950408889634 / (hd * hd));  // -log2(e) / h^2
    }
}

// The FP32 remainder of the Gaussian's FP64 scale after its FP32 value (the
// fine Gaussian uses t + tl).
float kernel_scale_lo(int kernel, float h)
{
    if (kernel != PI_KERNEL_GAUSSIAN) return 0.f;
    const double hd = (double)h, t = -1.4426950408889634 / (hd * hd);
    return (float)(t - (double)(float)t);
}

// Whether the scale of h is usable: finite for the Gaussian (below about
// h = 6.5e-20 it overflows FP32, and 0 * -inf would turn the term of two
// coincident particles into NaN), finite and non-zero for Lennard-Jones
// (sigma^2 = h^2 must neither overflow nor flush to zero).
bool scale_ok(int kernel, float h)
{
    const float t = kernel_scale(kernel, h);
    switch (kernel) {
        case PI_KERNEL_LJ:
        case PI_KERNEL_HIGHFLOP: return std::isfinite(t) && t > 0.f;
        case PI_KERNEL_LOWFLOP: return true;
        default: return std::isfinite(t);
    }
}

}  // namespace

namespace pi {
// Lets other translation units report a message through pi_last_error().
void set_last_error_text(const char* text)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s", text);
}
}  // namespace pi

extern "C" {

const char* pi_status_str(pi_status s)
{
    switch (s) {
        case PI_OK: return "ok";
        case PI_ERR_INVALID_ARG: return "invalid argument";
        case PI_ERR_CAPACITY: return "capacity exceeded";
        case PI_ERR_OUT_OF_BOX: return "position outside the box";
        case PI_ERR_NOT_BINNED: return "interaction requested before binning";
        case PI_ERR_CUDA: return "CUDA error";
        case PI_ERR_TIMEOUT: return "device-side wait timed out";
        case PI_ERR_NOMEM: return "device allocation failed";
        case PI_ERR_CHECK: return "bounds check failed (debug build)";
    }
    return "unknown status";
}

const char* pi_last_error(void) { return g_last_error; }

pi_status pi_batch_create(int32_t num_systems, const pi_box* boxes, const float* r_c,
                          const int64_t* n_max, pi_ctx** out)
{
    if (!out) return PI_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_systems < 1 || num_systems > pi::MAX_SYSTEMS || !boxes || !r_c || !n_max)
        return PI_ERR_INVALID_ARG;
    const int S = num_systems;
    pi_ctx* c = new (std::nothrow) pi_ctx();
    if (!c) return PI_ERR_NOMEM;
    c->S = S;
    c->boxes.assign(boxes, boxes + S);
    c->rc.assign(r_c, r_c + S);
    c->n_max.assign(n_max, n_max + S);
    c->sys.resize(S);
    c->cbase.assign(S + 1, 0);
    c->wbase.assign(S + 1, 0);
    c->rbase.assign(S + 1, 0);
    c->pbase_h.assign(S + 1, 0);
    c->kscale_h.assign(2 * (size_t)S, std::nanf(""));
    int64_t C = 0, N = 0, R = 0, RW = 0;
    for (int s = 0; s < S; ++s) {
        int64_t cells = 0;
        pi_status st = make_system(boxes[s], r_c[s], c->sys[s], cells);
        if (st == PI_OK && n_max[s] < 0) st = PI_ERR_INVALID_ARG;
        if (st != PI_OK) {
            delete c;
            return st;
        }
        SysDesc& d = c->sys[s];
        d.nseg = (uint32_t)((d.g.n[0] + pi::SEG_CELLS - 1) / pi::SEG_CELLS);
        d.cell_base = (uint32_t)C;
        d.work_base = (uint32_t)R;
        d.row_base = (uint32_t)RW;
        c->cbase[s] = (uint32_t)C;
        c->wbase[s] = (uint32_t)R;
        c->rbase[s] = (uint32_t)RW;
        C += cells;
        R += (int64_t)d.g.n[1] * d.g.n[2] * d.nseg;
        RW += (int64_t)d.g.n[1] * d.g.n[2];
        N += n_max[s];
        if (C >= ((int64_t)1 << 31) - 1 || N >= (int64_t)2147483647 - 64 || R >= ((int64_t)1 << 31)) {
            delete c;
            return PI_ERR_INVALID_ARG;
        }
    }
    c->cbase[S] = (uint32_t)C;
    c->wbase[S] = (uint32_t)R;
    c->rbase[S] = (uint32_t)RW;
    c->rows = RW;
    c->C = C;
    c->C_alloc = C;
    c->n_max_total = N;
    c->work = (uint32_t)R;
    c->algo = PI_ALGO_TILED;
    c->precision = PI_PREC_FP32;
    c->kernel = PI_KERNEL_GAUSSIAN;
    c->tile = PI_TILE_AUTO;
    c->wait_limit_ns = 1000000000ull;
    c->binning = PI_BIN_PER_PARTICLE;
    c->count_evals = 0;

    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = pi::tiled_occupancy(false, c->tiled_per_sm[0]);
    if (e == cudaSuccess) e = pi::tiled_occupancy(true, c->tiled_per_sm[1]);
    if (e != cudaSuccess) {
        pi_status st = cuda_fail(e, "pi_batch_create: device query");
        delete c;
        return st;
    }

    const size_t nm = (size_t)N;
    // the bucketed binning's count matrix: at most BUCKET_MAX buckets of at
    // least 32 cells by the chunks of n_max particles, capped at 4 M entries
    const size_t buckets_max = std::min<size_t>(pi::BUCKET_MAX, ((size_t)C + 31) / 32);
    const size_t chunks_max = std::max<size_t>(1, (nm + pi::BUCKET_CHUNK - 1) / pi::BUCKET_CHUNK);
    // (or the radix binning's digit x chunk matrix: up to 2^RADIX_MAX_BITS
    // digits by the chunks of n_max particles)
    const size_t radix_chunks = std::max<size_t>(1, (nm + pi::RADIX_CHUNK - 1) / pi::RADIX_CHUNK);
    const size_t mat_cap = std::max(std::min<size_t>((size_t)4 << 20, buckets_max * chunks_max + 1),
                                    ((size_t)1 << pi::RADIX_MAX_BITS) * radix_chunks + 1);
    const size_t tiles = (std::max<size_t>((size_t)C, mat_cap) + 1 + pi::SCAN_TILE - 1) / pi::SCAN_TILE;
    Carver k;
    const size_t o_ctrl = k.take<Ctrl>(1);
    const size_t o_counts = k.take<uint32_t>((size_t)C + 4);
    const size_t o_xbins = k.take<uint2>((size_t)C + 4);  // ctrl .. xbins: cleared by every pi_bin
    const size_t o_pbase = k.take<uint32_t>((size_t)S + 1);
    const size_t o_offsets = k.take<uint32_t>((size_t)C + 1 + 16);
    const size_t o_status = k.take<unsigned long long>(tiles);
    const size_t o_sys = k.take<SysDesc>((size_t)S);
    const size_t o_cbase = k.take<uint32_t>((size_t)S + 1);
    const size_t o_wbase = k.take<uint32_t>((size_t)S + 1);
    const size_t o_rbase = k.take<uint32_t>((size_t)S + 1);
    const size_t o_kscale = k.take<float>(2 * (size_t)S);
    const size_t o_partial = k.take<double>((size_t)S * pi::TOTAL_PARTS);
    const size_t o_ranges = k.take<uint32_t>(6 * (size_t)S);
    const size_t o_mat = k.take<uint32_t>(mat_cap);
    const size_t o_mat_base = k.take<uint32_t>(mat_cap + 1);
    const size_t o_ovf = k.take<uint2>(pi::BUCKET_MAX);
    const size_t o_cell = k.take<uint32_t>(nm + 4);
    const size_t o_rank = k.take<uint32_t>(nm + 4);
    const size_t o_rec = k.take<Rec>(nm + 4);
    const size_t o_perm = k.take<uint32_t>(nm + 4);
    const size_t o_sx = k.take<float>(nm + 4);
    const size_t o_sy = k.take<float>(nm + 4);
    const size_t o_sz = k.take<float>(nm + 4);
    // P: the particles plus ROW_PADS slots per X-row; rows <= cells for
    // every grid pi_reconfigure may set
    const size_t o_P = k.take<float4>(nm + (size_t)pi::ROW_PADS * (size_t)C + 8);
    const size_t total = align_up(k.off, 256);

    e = cudaMalloc(&c->arena, total);
    if (e != cudaSuccess) {
        pi_status st = cuda_fail(e, "pi_batch_create: cudaMalloc");
        delete c;
        return st;
    }
    char* base = (char*)c->arena;
    c->ctrl = (Ctrl*)(base + o_ctrl);
    c->counts = (uint32_t*)(base + o_counts);
    c->xbins = (uint2*)(base + o_xbins);
    c->pbase = (uint32_t*)(base + o_pbase);
    c->offsets = (uint32_t*)(base + o_offsets);
    c->scan_status = (unsigned long long*)(base + o_status);
    c->d_sys = (SysDesc*)(base + o_sys);
    c->d_cbase = (uint32_t*)(base + o_cbase);
    c->d_wbase = (uint32_t*)(base + o_wbase);
    c->d_rbase = (uint32_t*)(base + o_rbase);
    c->d_kscale = (float*)(base + o_kscale);
    c->d_partial = (double*)(base + o_partial);
    c->d_ranges = (uint32_t*)(base + o_ranges);
    c->mat = (uint32_t*)(base + o_mat);
    c->mat_base = (uint32_t*)(base + o_mat_base);
    c->ovf_list = (uint2*)(base + o_ovf);
    c->mat_cap = mat_cap;
    c->cell = (uint32_t*)(base + o_cell);
    c->rank = (uint32_t*)(base + o_rank);
    c->rec = (Rec*)(base + o_rec);
    c->perm = (uint32_t*)(base + o_perm);
    c->sx = (float*)(base + o_sx);
    c->sy = (float*)(base + o_sy);
    c->sz = (float*)(base + o_sz);
    c->P = (float4*)(base + o_P);
    // everything starts at zero: an empty grid, no error, stale-free scan
    // descriptors; then the per-system constants
    e = cudaMemset(c->arena, 0, total);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_sys, c->sys.data(), sizeof(SysDesc) * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_cbase, c->cbase.data(), sizeof(uint32_t) * (S + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_wbase, c->wbase.data(), sizeof(uint32_t) * (S + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(c->d_rbase, c->rbase.data(), sizeof(uint32_t) * (S + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        pi_status st = cuda_fail(e, "pi_batch_create: initialise");
        cudaFree(c->arena);
        delete c;
        return st;
    }
    *out = c;
    return PI_OK;
}

pi_status pi_create(const pi_box* box, float r_c, int64_t n_max, pi_ctx** out)
{
    if (!box || !out) return PI_ERR_INVALID_ARG;
    return pi_batch_create(1, box, &r_c, &n_max, out);
}

pi_status pi_destroy(pi_ctx* ctx)
{
    if (!ctx) return PI_OK;
    DeviceScope ds(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (ctx->io) cudaFree(ctx->io);
    cudaError_t e2 = cudaFree(ctx->arena);
    delete ctx;
    if (e != cudaSuccess) return cuda_fail(e, "pi_destroy: synchronize");
    if (e2 != cudaSuccess) return cuda_fail(e2, "pi_destroy: cudaFree");
    return PI_OK;
}

pi_status pi_reconfigure(pi_ctx* ctx, const pi_box* box, float r_c, pi_stream stream)
{
    if (!ctx || !box) return PI_ERR_INVALID_ARG;
    if (ctx->S != 1) return PI_ERR_INVALID_ARG;
    SysDesc d;
    int64_t cells = 0;
    const pi_status st = make_system(*box, r_c, d, cells);
    if (st != PI_OK) return st;
    if (cells > ctx->C_alloc) return PI_ERR_CAPACITY;
    d.nseg = (uint32_t)((d.g.n[0] + pi::SEG_CELLS - 1) / pi::SEG_CELLS);
    d.cell_base = 0;
    d.work_base = 0;
    d.row_base = 0;
    const int64_t work = (int64_t)d.g.n[1] * d.g.n[2] * d.nseg;
    const int64_t rows = (int64_t)d.g.n[1] * d.g.n[2];
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_reconfigure: set device");
    PI_TRY(pi::launch_set_system(ctx->d_sys, ctx->d_cbase, ctx->d_wbase, ctx->d_rbase, d, (uint32_t)cells,
                                 (uint32_t)work, (uint32_t)rows, (cudaStream_t)stream));
    ctx->launches += 1;
    ctx->boxes[0] = *box;
    ctx->rc[0] = r_c;
    ctx->sys[0] = d;
    ctx->cbase[1] = (uint32_t)cells;
    ctx->wbase[1] = (uint32_t)work;
    ctx->rbase[1] = (uint32_t)rows;
    ctx->rows = rows;
    ctx->C = cells;
    ctx->work = (uint32_t)work;
    ctx->binned = 0;
    std::fill(ctx->kscale_h.begin(), ctx->kscale_h.end(), std::nanf(""));
    return PI_OK;
}

pi_status pi_batch_info(const pi_ctx* ctx, int32_t* num_systems, int64_t* total_cells,
                        int64_t* total_n_max)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (num_systems) *num_systems = ctx->S;
    if (total_cells) *total_cells = ctx->C;
    if (total_n_max) *total_n_max = ctx->n_max_total;
    return PI_OK;
}

pi_status pi_batch_grid(const pi_ctx* ctx, int32_t system, int32_t dims[3])
{
    if (!ctx || !dims || system < 0 || system >= ctx->S) return PI_ERR_INVALID_ARG;
    for (int d = 0; d < 3; ++d) dims[d] = ctx->sys[system].g.n[d];
    return PI_OK;
}

pi_status pi_grid(const pi_ctx* ctx, int32_t dims[3]) { return pi_batch_grid(ctx, 0, dims); }

pi_status pi_batch_set_tiles(pi_ctx* ctx, const int32_t* tiles)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (!tiles) {
        ctx->sys_tile.clear();
        return PI_OK;
    }
    for (int s = 0; s < ctx->S; ++s)
        if (tiles[s] != 5 && tiles[s] != 6) return PI_ERR_INVALID_ARG;
    ctx->sys_tile.assign(tiles, tiles + ctx->S);
    return PI_OK;
}

pi_status pi_batch_tiles(const pi_ctx* ctx, int32_t* tiles)
{
    if (!ctx || !tiles) return PI_ERR_INVALID_ARG;
    for (int s = 0; s < ctx->S; ++s) tiles[s] = ctx->sys_tile.empty() ? -1 : ctx->sys_tile[s];
    return PI_OK;
}

pi_status pi_binned(const pi_ctx* ctx, const uint32_t** counts, const uint32_t** offsets,
                    const uint32_t** perm, const float** sx, const float** sy, const float** sz)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (counts) *counts = ctx->counts;
    if (offsets) *offsets = ctx->offsets;
    if (perm) *perm = ctx->perm;
    if (sx) *sx = ctx->sx;
    if (sy) *sy = ctx->sy;
    if (sz) *sz = ctx->sz;
    return PI_OK;
}

pi_status pi_copy_binned(const pi_ctx* ctx, uint32_t* counts, uint32_t* offsets, uint32_t* perm,
                         float* sx, float* sy, float* sz, pi_stream stream)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (!ctx->binned) return PI_ERR_NOT_BINNED;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_copy_binned: set device");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t C = (size_t)ctx->C, n = (size_t)ctx->n;
    const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    if (counts) PI_TRY(cudaMemcpyAsync(counts, ctx->counts, C * 4, k, s));
    if (offsets) PI_TRY(cudaMemcpyAsync(offsets, ctx->offsets, (C + 1) * 4, k, s));
    if (n > 0) {
        if (perm) PI_TRY(cudaMemcpyAsync(perm, ctx->perm, n * 4, k, s));
        if (sx) PI_TRY(cudaMemcpyAsync(sx, ctx->sx, n * 4, k, s));
        if (sy) PI_TRY(cudaMemcpyAsync(sy, ctx->sy, n * 4, k, s));
        if (sz) PI_TRY(cudaMemcpyAsync(sz, ctx->sz, n * 4, k, s));
    }
    return PI_OK;
}

pi_status pi_set_option(pi_ctx* ctx, int key, int64_t value)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    switch (key) {
        case PI_OPT_ALGO:
            if (value != PI_ALGO_TILED && value != PI_ALGO_PPNL) return PI_ERR_INVALID_ARG;
            ctx->algo = (int)value;
            return PI_OK;
        case PI_OPT_PRECISION:
            if (value != PI_PREC_FP32 && value != PI_PREC_KAHAN) return PI_ERR_INVALID_ARG;
            ctx->precision = (int)value;
            return PI_OK;
        case PI_OPT_WAIT_LIMIT_NS:
            if (value < 1000 || value > (int64_t)60000000000ll) return PI_ERR_INVALID_ARG;
            ctx->wait_limit_ns = (uint64_t)value;
            return PI_OK;
        case PI_OPT_TEST_WITHHOLD_SCAN:
            if (value != 0 && value != 1) return PI_ERR_INVALID_ARG;
            ctx->withhold_scan = (int)value;
            return PI_OK;
        case PI_OPT_TILE:
            if (value < PI_TILE_AUTO || value >= pi::NUM_TILES) return PI_ERR_INVALID_ARG;
            ctx->tile = (int)value;
            return PI_OK;
        case PI_OPT_BINNING:
            if (value != PI_BIN_PER_PARTICLE && value != PI_BIN_BUCKETED && value != PI_BIN_RADIX)
                return PI_ERR_INVALID_ARG;
            ctx->binning = (int)value;
            return PI_OK;
        case PI_OPT_COUNT_EVALS:
            if (value != 0 && value != 1) return PI_ERR_INVALID_ARG;
            ctx->count_evals = (int)value;
            return PI_OK;
        case PI_OPT_KERNEL:
            if (value < PI_KERNEL_GAUSSIAN || value > PI_KERNEL_HIGHFLOP) return PI_ERR_INVALID_ARG;
            ctx->kernel = (int)value;
            std::fill(ctx->kscale_h.begin(), ctx->kscale_h.end(), std::nanf(""));
            return PI_OK;
    }
    return PI_ERR_INVALID_ARG;
}

pi_status pi_launch_count(const pi_ctx* ctx, uint64_t* count)
{
    if (!ctx || !count) return PI_ERR_INVALID_ARG;
    *count = ctx->launches;
    return PI_OK;
}

pi_status pi_eval_count(pi_ctx* ctx, pi_stream stream, uint64_t* evaluations)
{
    if (!ctx || !evaluations) return PI_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_eval_count: set device");
    PI_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    unsigned long long v = 0;
    PI_TRY(cudaMemcpy(&v, &ctx->ctrl->evals, sizeof v, cudaMemcpyDeviceToHost));
    *evaluations = v;
    return PI_OK;
}

pi_status pi_batch_bin(pi_ctx* ctx, const float* x, const float* y, const float* z,
                       const int64_t* n, pi_stream stream)
{
    if (!ctx || !n) return PI_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int s = 0; s < ctx->S; ++s) {
        if (n[s] < 0) return PI_ERR_INVALID_ARG;
        if (n[s] > ctx->n_max[s]) return PI_ERR_CAPACITY;
        total += n[s];
    }
    if (total > 0 && (!x || !y || !z)) return PI_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_bin: set device");
    cudaStream_t s = (cudaStream_t)stream;
    ctx->binned = 0;
    ctx->tiled_seq = 0;  // k_zero clears both row-counter slots
    ctx->epoch = (ctx->epoch % 0x3ffffffeu) + 1u;  // 30-bit, never 0
    ctx->pbase_h[0] = 0;
    for (int k = 0; k < ctx->S; ++k) ctx->pbase_h[k + 1] = ctx->pbase_h[k] + (uint32_t)n[k];
    const uint32_t nn = (uint32_t)total;
    const uint32_t C = (uint32_t)ctx->C;
    pi::Systems sy{ctx->d_sys, ctx->pbase, ctx->d_cbase, ctx->d_wbase, ctx->d_rbase, ctx->S};

    pi::RadixPlan rp;
    if (ctx->binning == PI_BIN_RADIX && pi::radix_plan(nn, C, ctx->mat_cap, rp)) {
        // radix: per digit pass, a histogram per chunk (the first fused with
        // the cells), a scan of the digit x chunk matrix and a stable split;
        // the sorted keys then give offsets, perm and the sorted positions,
        // and a last pass counts, x-ranks and pads.  Every cell's count,
        // offset and sub-bin word is written, so only the control block is
        // cleared.  Keys and values ping-pong between (cell, rank) and the
        // record buffer; each scan takes its own epoch and ticket.
        uint32_t* keys[2] = {ctx->cell, reinterpret_cast<uint32_t*>(ctx->rec)};
        uint32_t* vals[2] = {ctx->rank, reinterpret_cast<uint32_t*>(ctx->rec) + ctx->n_max_total + 4};
        PI_TRY(pi::launch_zero((uint32_t*)ctx->ctrl, sizeof(Ctrl) / 4, ctx->pbase, ctx->pbase_h.data(), ctx->S + 1,
                               s));
        PI_TRY(pi::launch_radix_keys(x, y, z, nn, sy, rp, keys[0], ctx->mat, ctx->ctrl, s));
        const uint32_t entries = rp.bins * rp.chunks;
        for (uint32_t pass = 0; pass < rp.passes; ++pass) {
            const uint32_t shift = pass * rp.digit_bits;
            const int from = (int)(pass & 1u), to = from ^ 1;
            if (pass > 0) {
                PI_TRY(pi::launch_radix_count(keys[from], nn, rp, shift, ctx->mat, ctx->ctrl, s));
                ctx->epoch = (ctx->epoch % 0x3ffffffeu) + 1u;
            }
            PI_TRY(pi::launch_scan(ctx->mat, entries, ctx->mat_base, ctx->scan_status, ctx->ctrl, ctx->epoch,
                                   ctx->wait_limit_ns, pass == 0 ? ctx->withhold_scan : 0, s, 0, (int)pass));
            PI_TRY(pi::launch_radix_scatter(keys[from], pass == 0 ? nullptr : vals[from], keys[to], vals[to], nn, rp,
                                            shift, ctx->mat_base, ctx->ctrl, s));
        }
        const int fin = (int)(rp.passes & 1u);
        PI_TRY(pi::launch_radix_gather(keys[fin], vals[fin], x, y, z, nn, C, ctx->offsets, ctx->perm, ctx->sx,
                                       ctx->sy, ctx->sz, ctx->ctrl, ctx->num_sms, s));
        PI_TRY(pi::launch_radix_rank(keys[fin], nn, sy, C, ctx->offsets, ctx->perm, ctx->sx, ctx->sy, ctx->sz,
                                     ctx->counts, ctx->P, ctx->xbins, ctx->ctrl, ctx->num_sms, s));
        ctx->launches += 3 * rp.passes + 3;  // zero, keys, per pass (count,) scan, split, gather, rank
        ctx->n = total;
        ctx->binned = 1;
        return PI_OK;
    }

    pi::BucketPlan plan;
    if (ctx->binning == PI_BIN_BUCKETED && pi::bucket_plan(nn, C, ctx->mat_cap, plan)) {
        // bucketed: count per chunk and bucket, scan the count matrix,
        // scatter to buckets, rank each bucket's cells in shared memory (and
        // the buckets too large for it grid-wide); every cell's count,
        // offset and sub-bin word is written, so only the control block is
        // cleared
        float4* rec = reinterpret_cast<float4*>(ctx->rec);
        float4* rec2 = rec + ctx->n_max_total;
        PI_TRY(pi::launch_zero((uint32_t*)ctx->ctrl, sizeof(Ctrl) / 4, ctx->pbase, ctx->pbase_h.data(), ctx->S + 1,
                               s));
        PI_TRY(pi::launch_bucket_count(x, y, z, nn, sy, plan, ctx->mat, ctx->ctrl, s));
        PI_TRY(pi::launch_scan(ctx->mat, plan.B * plan.chunks, ctx->mat_base, ctx->scan_status, ctx->ctrl,
                               ctx->epoch, ctx->wait_limit_ns, ctx->withhold_scan, s, 0));
        PI_TRY(pi::launch_bucket_scatter(x, y, z, nn, sy, plan, ctx->mat_base, rec, ctx->ctrl, s));
        PI_TRY(pi::launch_bucket_cells(rec, nn, sy, plan, ctx->mat_base, ctx->counts, ctx->offsets, ctx->perm,
                                       ctx->sx, ctx->sy, ctx->sz, ctx->P, ctx->xbins, rec2, ctx->ovf_list,
                                       ctx->ctrl, s));
        PI_TRY(pi::launch_bucket_big(rec2, nn, sy, plan, ctx->offsets, ctx->perm, ctx->sx, ctx->sy, ctx->sz, ctx->P,
                                     ctx->xbins, ctx->ovf_list, ctx->ctrl, ctx->num_sms, s));
        ctx->launches += 6;
        ctx->n = total;
        ctx->binned = 1;
        return PI_OK;
    }

    // per particle: control block, counts and xbins are one contiguous
    // zeroed prefix of the
    // arena; the same launch writes this step's particle bases
    const size_t zero_words = ((char*)(ctx->xbins + C) - (char*)ctx->ctrl + 3) / 4;
    PI_TRY(pi::launch_zero((uint32_t*)ctx->ctrl, zero_words, ctx->pbase, ctx->pbase_h.data(),
                           ctx->S + 1, s));
    ctx->launches += 1;
    if (nn > 0) {
        PI_TRY(pi::launch_hist(x, y, z, nn, sy, ctx->counts, ctx->cell, ctx->rank, ctx->ctrl,
                               ctx->num_sms, s));
        ctx->launches += 1;
    }
    PI_TRY(pi::launch_scan(ctx->counts, C, ctx->offsets, ctx->scan_status, ctx->ctrl, ctx->epoch,
                           ctx->wait_limit_ns, ctx->withhold_scan, s));
    ctx->launches += 1;
    if (nn > 0) {
        PI_TRY(pi::launch_scatter(ctx->cell, ctx->rank, x, y, z, nn, sy, ctx->offsets, ctx->rec,
                                  ctx->ctrl, ctx->num_sms, s));
        PI_TRY(pi::launch_stabilise(ctx->rec, nn, sy, ctx->offsets, ctx->perm, ctx->sx,
                                    ctx->sy, ctx->sz, ctx->P, ctx->xbins, ctx->ctrl, ctx->num_sms,
                                    s));
        ctx->launches += 2;
    }
    ctx->n = total;
    ctx->binned = 1;
    return PI_OK;
}

pi_status pi_bin(pi_ctx* ctx, const float* x, const float* y, const float* z, int64_t n,
                 pi_stream stream)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (ctx->S != 1) return PI_ERR_INVALID_ARG;
    return pi_batch_bin(ctx, x, y, z, &n, stream);
}

}  // extern "C"

namespace {

// The P ranges (row pads included) of the systems whose shape in
// ctx->sys_tile is `tile`, merged where consecutive systems share it, with
// the first block of each range for groups of `per` slots; returns the
// blocks of the list.  Systems without particles store nothing and are
// left out.
unsigned plan_ranges(const pi_ctx* ctx, int tile, uint32_t per, uint32_t* words, uint32_t* rblock, int& nr)
{
    nr = 0;
    for (int s = 0; s < ctx->S; ++s) {
        if (ctx->sys_tile[s] != tile || ctx->pbase_h[s + 1] == ctx->pbase_h[s]) continue;
        const uint32_t b = ctx->pbase_h[s] + pi::ROW_PADS * ctx->rbase[s];
        const uint32_t e = ctx->pbase_h[s + 1] + pi::ROW_PADS * ctx->rbase[s + 1];
        if (nr > 0 && words[2 * nr - 1] == b) {
            words[2 * nr - 1] = e;
        } else {
            words[2 * nr] = b;
            words[2 * nr + 1] = e;
            ++nr;
        }
    }
    unsigned blocks = 0;
    const uint32_t span = per * (uint32_t)pi::DIRECT_BLOCK;
    for (int r = 0; r < nr; ++r) {
        rblock[r] = blocks;
        blocks += (words[2 * r + 1] - words[2 * r] + span - 1) / span;
    }
    return blocks;
}

// The interaction of a batch under a per-system shape plan: one launch of
// each direct shape that some system uses, over its systems' P ranges.
pi_status launch_plan(pi_ctx* ctx, pi::InteractArgs a, bool kahan, cudaStream_t st, int* launched)
{
    const size_t S = (size_t)ctx->S;
    std::vector<uint32_t> w(6 * S, 0u);
    int nr5 = 0, nr6 = 0;
    const unsigned b5 = plan_ranges(ctx, 5, 2u, w.data(), w.data() + 4 * S, nr5);
    const unsigned b6 = plan_ranges(ctx, 6, 4u, w.data() + 2 * S, w.data() + 5 * S, nr6);
    if (w != ctx->ranges_h) {
        PI_TRY(pi::launch_write_words(ctx->d_ranges, w.data(), w.size(), st));
        *launched += (int)((w.size() + 4095) / 4096);
        ctx->ranges_h = w;
    }
    cudaError_t e = cudaSuccess;
    if (nr5 > 0) {
        a.ranges = reinterpret_cast<const uint2*>(ctx->d_ranges);
        a.rblock = ctx->d_ranges + 4 * S;
        a.nranges = nr5;
        a.range_blocks = b5;
        e = pi::launch_interact_tiled(a, kahan, ctx->num_sms, ctx->tiled_per_sm[kahan ? 1 : 0], 5, st, launched);
    }
    if (e == cudaSuccess && nr6 > 0) {
        a.ranges = reinterpret_cast<const uint2*>(ctx->d_ranges + 2 * S);
        a.rblock = ctx->d_ranges + 5 * S;
        a.nranges = nr6;
        a.range_blocks = b6;
        e = pi::launch_interact_tiled(a, kahan, ctx->num_sms, ctx->tiled_per_sm[kahan ? 1 : 0], 6, st, launched);
    }
    if (e != cudaSuccess) return cuda_fail(e, "pi_interact: launch");
    return PI_OK;
}

// Occupancy regimes of the per-system autotuning: mean particles per cell
// below 4, below 8, and from 8 on (the shapes' crossover is near 8).
int occupancy_regime(const pi_ctx* ctx, int s)
{
    const double cells = (double)ctx->cbase[s + 1] - (double)ctx->cbase[s];
    const double q = (double)(ctx->pbase_h[s + 1] - ctx->pbase_h[s]) / (cells > 0 ? cells : 1.0);
    return q < 4.0 ? 0 : (q < 8.0 ? 1 : 2);
}

}  // namespace

extern "C" {

pi_status pi_batch_interact(pi_ctx* ctx, const float* h, float* S, float* Vx, float* Vy, float* Vz,
                            uint32_t* nbr, int out_order, pi_stream stream)
{
    if (!ctx || !h) return PI_ERR_INVALID_ARG;
    for (int s = 0; s < ctx->S; ++s) {
        if (!(h[s] > 0.0f) || std::isinf(h[s])) return PI_ERR_INVALID_ARG;
        if (!scale_ok(ctx->kernel, h[s])) {
            std::snprintf(g_last_error, sizeof g_last_error,
                          "pi_interact: h = %g of system %d gives no finite FP32 kernel scale", (double)h[s], s);
            return PI_ERR_INVALID_ARG;
        }
    }
    if (out_order != PI_ORDER_SORTED && out_order != PI_ORDER_ORIGINAL) return PI_ERR_INVALID_ARG;
    if (!ctx->binned) return PI_ERR_NOT_BINNED;
    if (ctx->n > 0 && (!S || !Vx || !Vy || !Vz)) return PI_ERR_INVALID_ARG;
    if (ctx->n == 0) return PI_OK;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_interact: set device");
    cudaStream_t st = (cudaStream_t)stream;

    pi::InteractArgs a{};
    a.sy = pi::Systems{ctx->d_sys, ctx->pbase, ctx->d_cbase, ctx->d_wbase, ctx->d_rbase, ctx->S};
    a.P = ctx->P;
    a.xbins = ctx->xbins;
    a.sx = ctx->sx;
    a.sy_pos = ctx->sy;
    a.sz = ctx->sz;
    a.offsets = ctx->offsets;
    a.perm = ctx->perm;
    a.n = (uint32_t)ctx->n;
    a.np = (uint32_t)(ctx->n + pi::ROW_PADS * ctx->rows);
    a.work = ctx->work;
    a.one = 1.0f;
    a.zero = 0.0f;
    // the Gaussian with the compensated exponent where some system's kernel
    // is short next to its cutoff (r_c^2 / h^2 above FINE_GAUSS_RATIO)
    bool fine = false;
    if (ctx->kernel == PI_KERNEL_GAUSSIAN)
        for (int s = 0; s < ctx->S; ++s) {
            const double r = (double)ctx->rc[s] / (double)h[s];
            fine = fine || r * r > pi::FINE_GAUSS_RATIO;
        }
    a.kernel = fine ? pi::KERNEL_GAUSSIAN_FINE : ctx->kernel;
    if (ctx->S == 1) {
        a.kscale = nullptr;
        a.kscale0 = kernel_scale(ctx->kernel, h[0]);
        a.kscale0_lo = kernel_scale_lo(ctx->kernel, h[0]);
    } else {
        // write the per-system scales only when they changed
        const int S = ctx->S;
        bool same = true;
        std::vector<float> t(2 * (size_t)S);
        for (int s = 0; s < S; ++s) {
            t[s] = kernel_scale(ctx->kernel, h[s]);
            t[S + s] = kernel_scale_lo(ctx->kernel, h[s]);
        }
        for (int i = 0; i < 2 * S; ++i) same = same && t[i] == ctx->kscale_h[i];
        if (!same) {
            PI_TRY(pi::launch_set_kscale(ctx->d_kscale, t.data(), 2 * S, st));
            ctx->launches += 1;
            ctx->kscale_h = t;
        }
        a.kscale = ctx->d_kscale;
    }
    a.S = S;
    a.Vx = Vx;
    a.Vy = Vy;
    a.Vz = Vz;
    a.nbr = nbr;
    a.original_order = out_order == PI_ORDER_ORIGINAL;
    a.ctrl = ctx->ctrl;
    a.wait_limit_ns = ctx->wait_limit_ns;
    a.seq = ctx->tiled_seq;
    a.count_evals = ctx->count_evals;
    int launched = 0;
    cudaError_t e;
    const bool kahan = ctx->precision == PI_PREC_KAHAN;
    if (ctx->algo == PI_ALGO_PPNL) {
        e = pi::launch_interact_ppnl(a, kahan, ctx->num_sms, st, &launched);
    } else if (!ctx->sys_tile.empty()) {
        const pi_status ps = launch_plan(ctx, a, kahan, st, &launched);
        ctx->launches += (uint64_t)launched;
        ctx->tiled_seq += 1;
        return ps;
    } else {
        // PI_TILE_AUTO: four targets per thread for the plain Gaussian and
        // low-FLOP sums from 8 particles per cell on average (measured
        // faster from there on, slower below) when the four-target grid
        // fills at least one wave of the GPU (5 CTAs of 128 threads per SM);
        // two otherwise: a smaller grid leaves SMs idle and each thread twice
        // the work (measured 2x slower at 32,768 particles), and the
        // four-target Lennard-Jones and 168-FLOP forms (measured slower at 8
        // per cell) and the compensated sums keep all their registers and
        // run fewer warps
        constexpr int64_t QUAD_THREADS_PER_SM = 5 * 128;
        const bool packed =
            !kahan && ((ctx->kernel == PI_KERNEL_GAUSSIAN && !fine) || ctx->kernel == PI_KERNEL_LOWFLOP);
        const bool full_wave = ctx->n / 4 >= (int64_t)ctx->num_sms * QUAD_THREADS_PER_SM;
        const int tile = ctx->tile >= 0 ? ctx->tile
                         : (packed && full_wave && ctx->n >= 8 * ctx->C ? pi::HIGH_OCCUPANCY_TILE
                                                                         : pi::DEFAULT_TILE);
        e = pi::launch_interact_tiled(a, kahan, ctx->num_sms, ctx->tiled_per_sm[kahan ? 1 : 0], tile, st,
                                      &launched);
        ctx->tiled_seq += 1;
    }
    ctx->launches += (uint64_t)launched;
    if (e != cudaSuccess) return cuda_fail(e, "pi_interact: launch");
    return PI_OK;
}

pi_status pi_autotune(pi_ctx* ctx, const float* h, float* S, float* Vx, float* Vy, float* Vz,
                      uint32_t* nbr, int out_order, int reps, int32_t* chosen, float* ms,
                      pi_stream stream)
{
    if (!ctx || !h || reps < 1 || reps > 100) return PI_ERR_INVALID_ARG;
    if (!ctx->binned) return PI_ERR_NOT_BINNED;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_autotune: set device");
    cudaStream_t st = (cudaStream_t)stream;
    const int saved_algo = ctx->algo, saved_tile = ctx->tile, saved_count = ctx->count_evals;
    const std::vector<int> saved_plan = ctx->sys_tile;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PI_TRY(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ce, "pi_autotune: event");
    }
    pi_status result = PI_OK;
    ctx->count_evals = 0;  // the trials time the ordinary kernels and count nothing
    // median milliseconds of the interaction as the context stands: one
    // untimed run, then `reps` timed ones
    auto median_ms = [&](float& med) {
        result = pi_batch_interact(ctx, h, S, Vx, Vy, Vz, nbr, out_order, stream);
        std::vector<float> times;
        for (int r = 0; r < reps && result == PI_OK; ++r) {
            ce = cudaEventRecord(e0, st);
            if (ce == cudaSuccess) result = pi_batch_interact(ctx, h, S, Vx, Vy, Vz, nbr, out_order, stream);
            if (ce == cudaSuccess && result == PI_OK) ce = cudaEventRecord(e1, st);
            if (ce == cudaSuccess && result == PI_OK) ce = cudaEventSynchronize(e1);
            float m = 0.f;
            if (ce == cudaSuccess && result == PI_OK) ce = cudaEventElapsedTime(&m, e0, e1);
            if (ce != cudaSuccess && result == PI_OK) result = cuda_fail(ce, "pi_autotune: timing");
            times.push_back(m);
        }
        if (result != PI_OK) return false;
        std::sort(times.begin(), times.end());
        med = times[times.size() / 2];
        return true;
    };
    // candidates: every tile shape of the tiled algorithm, then Alg. 1, then
    // (batches) a shape per occupancy regime
    constexpr int PPNL = pi::NUM_TILES, REGIMES = pi::NUM_TILES + 1;
    float best = 0.f;
    int best_c = -1;
    ctx->sys_tile.clear();
    for (int t = 0; t <= PPNL && result == PI_OK; ++t) {
        ctx->algo = t == PPNL ? PI_ALGO_PPNL : PI_ALGO_TILED;
        if (t < PPNL) ctx->tile = t;
        float med = 0.f;
        if (!median_ms(med)) break;
        if (ms) ms[t] = med;
        if (best_c < 0 || med < best) {
            best = med;
            best_c = t;
        }
    }
    if (ms) ms[REGIMES] = 0.f;
    std::vector<int> plan;
    if (result == PI_OK && ctx->S > 1) {
        // per regime, the faster direct shape on its systems alone
        ctx->algo = PI_ALGO_TILED;
        plan.assign(ctx->S, 0);
        for (int g = 0; g < 3 && result == PI_OK; ++g) {
            std::vector<int> trial(ctx->S, 0);
            bool any = false;
            for (int s = 0; s < ctx->S; ++s)
                if (occupancy_regime(ctx, s) == g && ctx->pbase_h[s + 1] > ctx->pbase_h[s]) any = true;
            if (!any) continue;
            float tm[2] = {0.f, 0.f};
            for (int k = 0; k < 2 && result == PI_OK; ++k) {
                for (int s = 0; s < ctx->S; ++s) trial[s] = occupancy_regime(ctx, s) == g ? 5 + k : 0;
                ctx->sys_tile = trial;
                median_ms(tm[k]);
            }
            for (int s = 0; s < ctx->S; ++s)
                if (occupancy_regime(ctx, s) == g) plan[s] = tm[1] < tm[0] ? 6 : 5;
        }
        for (int s = 0; s < ctx->S; ++s)
            if (plan[s] == 0) plan[s] = 5;  // systems without particles
        float med = 0.f;
        ctx->sys_tile = plan;
        if (result == PI_OK && median_ms(med)) {
            if (ms) ms[REGIMES] = med;
            if (med < best) {
                best = med;
                best_c = REGIMES;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->count_evals = saved_count;
    if (result != PI_OK || best_c < 0) {
        ctx->algo = saved_algo;
        ctx->tile = saved_tile;
        ctx->sys_tile = saved_plan;
        return result;
    }
    ctx->algo = best_c == PPNL ? PI_ALGO_PPNL : PI_ALGO_TILED;
    ctx->tile = (best_c == PPNL || best_c == REGIMES) ? saved_tile : best_c;
    if (best_c == REGIMES)
        ctx->sys_tile = plan;
    else
        ctx->sys_tile.clear();
    if (chosen) *chosen = best_c;
    // the outputs of the chosen configuration (the last trial may have left
    // some systems out)
    return pi_batch_interact(ctx, h, S, Vx, Vy, Vz, nbr, out_order, stream);
}

pi_status pi_interact(pi_ctx* ctx, float h, float* S, float* Vx, float* Vy, float* Vz,
                      uint32_t* nbr, int out_order, pi_stream stream)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (ctx->S != 1) return PI_ERR_INVALID_ARG;
    return pi_batch_interact(ctx, &h, S, Vx, Vy, Vz, nbr, out_order, stream);
}

pi_status pi_total_f64(pi_ctx* ctx, const float* v, double* out, pi_stream stream)
{
    if (!ctx || !out) return PI_ERR_INVALID_ARG;
    if (!ctx->binned) return PI_ERR_NOT_BINNED;
    if (ctx->n > 0 && !v) return PI_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_total_f64: set device");
    pi::Systems sy{ctx->d_sys, ctx->pbase, ctx->d_cbase, ctx->d_wbase, ctx->d_rbase, ctx->S};
    PI_TRY(pi::launch_total_f64(ctx->n > 0 ? v : ctx->sx, sy, ctx->d_partial, pi::TOTAL_PARTS, out,
                                (cudaStream_t)stream));
    ctx->launches += 2;
    return PI_OK;
}

pi_status pi_sync_status(pi_ctx* ctx, pi_stream stream, uint32_t* max_per_cell)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_sync_status: set device");
    PI_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    Ctrl h{};
    PI_TRY(cudaMemcpy(&h, ctx->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    if (max_per_cell) *max_per_cell = h.max_per_cell;
    if (h.error & pi::ERR_CHECK) {
        std::snprintf(g_last_error, sizeof g_last_error, "bounds check failed at site %u (see CheckSite)",
                      h.check_site);
        return PI_ERR_CHECK;
    }
    if (h.error & pi::ERR_TIMEOUT) return PI_ERR_TIMEOUT;
    if (h.error & pi::ERR_OUT_OF_BOX) return PI_ERR_OUT_OF_BOX;
    if (h.error & pi::ERR_CAPACITY) return PI_ERR_CAPACITY;
    return PI_OK;
}

// Entries per staging array of a context (its particle capacity, rounded).
static size_t io_entries(const pi_ctx* ctx)
{
    return ((size_t)ctx->n_max_total + 4 + 3) & ~(size_t)3;
}

// Device staging buffers of the host-memory entry points (allocated on the
// first call: io_entries entries for each of x, y, z, S, Vx, Vy, Vz, nbr).
static pi_status ensure_io(pi_ctx* ctx)
{
    if (ctx->io) return PI_OK;
    const size_t nm = io_entries(ctx);
    PI_TRY(cudaMalloc(&ctx->io, nm * 8 * sizeof(float)));
    ctx->io_n = nm;
    return PI_OK;
}

// The asynchronous body of pi_run_host / pi_submit_host /
// pi_submit_host_strided.  in_stride / out_stride: 0 for separate host
// arrays (one copy each), else the stride (elements) of host arrays that
// lie in one block (one copy per block, the gaps included); the device
// staging arrays take the same stride.
static pi_status host_step(pi_ctx* ctx, const float* hx, const float* hy, const float* hz,
                           size_t in_stride, int64_t n, float h, float* hS, float* hVx, float* hVy,
                           float* hVz, uint32_t* hnbr, size_t out_stride, int out_order, pi_stream stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * sizeof(float), nm = ctx->io_n;
    float* dx = ctx->io;
    const size_t si = in_stride ? in_stride : nm;
    if (n > 0) {
        if (in_stride) {
            PI_TRY(cudaMemcpyAsync(dx, hx, (2 * si + (size_t)n) * sizeof(float), cudaMemcpyHostToDevice, s));
        } else {
            PI_TRY(cudaMemcpyAsync(dx, hx, bytes, cudaMemcpyHostToDevice, s));
            PI_TRY(cudaMemcpyAsync(dx + nm, hy, bytes, cudaMemcpyHostToDevice, s));
            PI_TRY(cudaMemcpyAsync(dx + 2 * nm, hz, bytes, cudaMemcpyHostToDevice, s));
        }
    }
    pi_status st = pi_bin(ctx, dx, dx + si, dx + 2 * si, n, stream);
    if (st != PI_OK) return st;
    float* d0 = ctx->io + 3 * nm;
    const size_t so = out_stride ? out_stride : nm;
    st = pi_interact(ctx, h, d0, d0 + so, d0 + 2 * so, d0 + 3 * so, hnbr ? (uint32_t*)(d0 + 4 * so) : nullptr,
                     out_order, stream);
    if (st != PI_OK) return st;
    if (n > 0) {
        if (out_stride) {
            const size_t k = hnbr ? 5 : 4;
            PI_TRY(cudaMemcpyAsync(hS, d0, ((k - 1) * so + (size_t)n) * sizeof(float), cudaMemcpyDeviceToHost, s));
        } else {
            PI_TRY(cudaMemcpyAsync(hS, d0, bytes, cudaMemcpyDeviceToHost, s));
            PI_TRY(cudaMemcpyAsync(hVx, d0 + nm, bytes, cudaMemcpyDeviceToHost, s));
            PI_TRY(cudaMemcpyAsync(hVy, d0 + 2 * nm, bytes, cudaMemcpyDeviceToHost, s));
            PI_TRY(cudaMemcpyAsync(hVz, d0 + 3 * nm, bytes, cudaMemcpyDeviceToHost, s));
            if (hnbr) PI_TRY(cudaMemcpyAsync(hnbr, d0 + 4 * nm, bytes, cudaMemcpyDeviceToHost, s));
        }
    }
    return PI_OK;
}

// Re-targets a single-system context to another box and cutoff unless it
// already has them.
static pi_status retarget(pi_ctx* ctx, const pi_box* box, float r_c, pi_stream stream)
{
    const pi_box& cur = ctx->boxes[0];
    bool same = r_c == ctx->rc[0];
    for (int d = 0; d < 3; ++d) same = same && box->lo[d] == cur.lo[d] && box->hi[d] == cur.hi[d];
    return same ? PI_OK : pi_reconfigure(ctx, box, r_c, stream);
}

static pi_status host_args_ok(const pi_ctx* ctx, const float* hx, const float* hy, const float* hz,
                              int64_t n, const float* hS, const float* hVx, const float* hVy,
                              const float* hVz)
{
    if (!ctx) return PI_ERR_INVALID_ARG;
    if (ctx->S != 1) return PI_ERR_INVALID_ARG;
    if (n < 0) return PI_ERR_INVALID_ARG;
    if (n > ctx->n_max[0]) return PI_ERR_CAPACITY;
    if (n > 0 && (!hx || !hy || !hz || !hS || !hVx || !hVy || !hVz)) return PI_ERR_INVALID_ARG;
    return PI_OK;
}

pi_status pi_run_host(pi_ctx* ctx, const float* hx, const float* hy, const float* hz, int64_t n,
                      float h, float* hS, float* hVx, float* hVy, float* hVz, uint32_t* hnbr,
                      int out_order, pi_stream stream)
{
    pi_status st = host_args_ok(ctx, hx, hy, hz, n, hS, hVx, hVy, hVz);
    if (st != PI_OK) return st;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_run_host: set device");
    if ((st = ensure_io(ctx)) != PI_OK) return st;
    st = host_step(ctx, hx, hy, hz, 0, n, h, hS, hVx, hVy, hVz, hnbr, 0, out_order, stream);
    if (st != PI_OK) return st;
    return pi_sync_status(ctx, stream, nullptr);
}

pi_status pi_submit_host(pi_ctx* ctx, const pi_box* box, float r_c, const float* hx, const float* hy,
                         const float* hz, int64_t n, float h, float* hS, float* hVx, float* hVy,
                         float* hVz, uint32_t* hnbr, int out_order, pi_stream stream)
{
    pi_status st = host_args_ok(ctx, hx, hy, hz, n, hS, hVx, hVy, hVz);
    if (st != PI_OK) return st;
    if (!box) return PI_ERR_INVALID_ARG;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_submit_host: set device");
    if ((st = ensure_io(ctx)) != PI_OK) return st;
    if ((st = retarget(ctx, box, r_c, stream)) != PI_OK) return st;
    return host_step(ctx, hx, hy, hz, 0, n, h, hS, hVx, hVy, hVz, hnbr, 0, out_order, stream);
}

pi_status pi_submit_host_strided(pi_ctx* ctx, const pi_box* box, float r_c, const float* hx, const float* hy,
                                 const float* hz, int64_t in_stride, int64_t n, float h, float* hS, float* hVx,
                                 float* hVy, float* hVz, uint32_t* hnbr, int64_t out_stride, int out_order,
                                 pi_stream stream)
{
    if (!ctx || !box) return PI_ERR_INVALID_ARG;
    const uint64_t cap = io_entries(ctx);
    auto stride_ok = [&](int64_t d) { return d == 0 || (d >= n && d % 4 == 0 && (uint64_t)d <= cap); };
    if (n < 0 || !stride_ok(in_stride) || !stride_ok(out_stride)) return PI_ERR_INVALID_ARG;
    // arrays of a block must sit at the stride they claim
    if (in_stride && (hy != hx + in_stride || hz != hx + 2 * in_stride)) return PI_ERR_INVALID_ARG;
    if (out_stride && (hVx != hS + out_stride || hVy != hS + 2 * out_stride || hVz != hS + 3 * out_stride ||
                       (hnbr && (const void*)hnbr != (const void*)(hS + 4 * out_stride))))
        return PI_ERR_INVALID_ARG;
    pi_status st = host_args_ok(ctx, hx, hy, hz, n, hS, hVx, hVy, hVz);
    if (st != PI_OK) return st;
    DeviceScope ds(ctx->device);
    if (ds.err != cudaSuccess) return cuda_fail(ds.err, "pi_submit_host_strided: set device");
    if ((st = ensure_io(ctx)) != PI_OK) return st;
    if ((st = retarget(ctx, box, r_c, stream)) != PI_OK) return st;
    return host_step(ctx, hx, hy, hz, (size_t)in_stride, n, h, hS, hVx, hVy, hVz, hnbr, (size_t)out_stride,
                     out_order, stream);
}

}  // extern "C"
