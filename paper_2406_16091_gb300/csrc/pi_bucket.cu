// pi_bucket.cu -- binning (a1-a4 of Sec. 2) by buckets of consecutive cells.
//
// The same results as the per-particle path of pi_bin.cu (counts, offsets,
// the stable permutation, the sorted SoA, the row-padded x-ordered copy P
// and each cell's sub-bin starts, bit for bit), computed without one global
// atomic per particle and without 32-byte records scattered one by one:
//
//   k_bucket_count    per chunk of input particles, a shared-memory
//                     histogram of the buckets (2^k consecutive cells) its
//                     particles fall in, written as one column of the
//                     bucket x chunk count matrix
//   k_scan            (pi_bin.cu) the exclusive scan of that matrix in
//                     bucket-major order: where each chunk's particles of
//                     each bucket start, and where each bucket starts
//   k_bucket_scatter  per chunk, each particle to its bucket as a 16-byte
//                     record (x, y, z, input index); inside a (bucket,
//                     chunk) run the order is that of shared atomics
//   k_bucket_cells    one CTA per bucket: loads the bucket's records into
//                     shared memory, counts and scans its cells (offsets of
//                     Fig. 1 = bucket start + local prefix), sorts the
//                     records by cell, and per particle counts the members
//                     of its cell with a smaller input index (the stable
//                     rank: input order inside a cell) and with a smaller x
//                     (the x-rank of P), as the per-particle path does from
//                     its provisional records
//   k_bucket_big      buckets of more than BUCKET_CAP particles (dense
//                     clusters): k_bucket_cells only counts, scans and puts
//                     their records in cell order; this grid-wide kernel
//                     ranks them, one thread per particle
#include <algorithm>
#include <mutex>

#include "pi_internal.cuh"

namespace pi {

namespace {

constexpr int CHUNK_THREADS = 512;
constexpr int GROUPS = 2;  // groups of four particles a chunk thread has in flight
constexpr int CELL_THREADS = 256;
constexpr unsigned long long OVF_MASK = (1ull << 40) - 1ull;

__global__ void __launch_bounds__(CHUNK_THREADS, 2) k_bucket_count(const float* __restrict__ x,
                                                                const float* __restrict__ y,
                                                                const float* __restrict__ z, uint32_t n,
                                                                Systems sy, BucketPlan plan, uint32_t chunk,
                                                                uint32_t* __restrict__ mat, Ctrl* __restrict__ ctrl,
                                                                int vec)
{
    extern __shared__ uint32_t hist[];
    pdl_trigger();
    for (uint32_t b = threadIdx.x; b < plan.B; b += CHUNK_THREADS) hist[b] = 0u;
    __syncthreads();
    pdl_wait();  // the particle bases and the control block are k_zero's
    const uint32_t k = blockIdx.x;
    const uint32_t beg = k * chunk, end = min(beg + chunk, n);
    bool ok = true;
    for (uint32_t i0 = beg + 4u * threadIdx.x; i0 < end; i0 += 4u * CHUNK_THREADS * GROUPS) {
        // GROUPS groups of four in flight before the first atomic
        float px[GROUPS][4], py[GROUPS][4], pz[GROUPS][4];
        bool valid[GROUPS][4];
#pragma unroll
        for (int g = 0; g < GROUPS; ++g)
            load4(x, y, z, i0 + 4u * CHUNK_THREADS * g, end, vec, px[g], py[g], pz[g], valid[g]);
#pragma unroll
        for (int g = 0; g < GROUPS; ++g) {
            uint32_t cell[4];
            cells4(sy, i0 + 4u * CHUNK_THREADS * g, px[g], py[g], pz[g], valid[g], cell, ok);
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (valid[g][j] && PI_BOUNDS(ctrl, cell[j] >> plan.bc_log2, plan.B, CS_HIST_COUNTS))
                    atomicAdd(&hist[cell[j] >> plan.bc_log2], 1u);
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < plan.B; b += CHUNK_THREADS) mat[(size_t)b * plan.chunks + k] = hist[b];
    if (!ok) atomicOr(&ctrl->error, ERR_OUT_OF_BOX);
}

__global__ void __launch_bounds__(CHUNK_THREADS, 2) k_bucket_scatter(const float* __restrict__ x,
                                                                  const float* __restrict__ y,
                                                                  const float* __restrict__ z, uint32_t n,
                                                                  Systems sy, BucketPlan plan, uint32_t chunk,
                                                                  const uint32_t* __restrict__ base,
                                                                  float4* __restrict__ rec, Ctrl* __restrict__ ctrl,
                                                                  int vec)
{
    extern __shared__ uint32_t cur[];
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    const uint32_t k = blockIdx.x;
    for (uint32_t b = threadIdx.x; b < plan.B; b += CHUNK_THREADS) cur[b] = base[(size_t)b * plan.chunks + k];
    __syncthreads();
    const uint32_t beg = k * chunk, end = min(beg + chunk, n);
    bool ok = true;
    for (uint32_t i0 = beg + 4u * threadIdx.x; i0 < end; i0 += 4u * CHUNK_THREADS * GROUPS) {
        float px[GROUPS][4], py[GROUPS][4], pz[GROUPS][4];
        bool valid[GROUPS][4];
#pragma unroll
        for (int g = 0; g < GROUPS; ++g)
            load4(x, y, z, i0 + 4u * CHUNK_THREADS * g, end, vec, px[g], py[g], pz[g], valid[g]);
#pragma unroll
        for (int g = 0; g < GROUPS; ++g) {
            const uint32_t ig = i0 + 4u * CHUNK_THREADS * g;
            uint32_t cell[4], slot[4];
            cells4(sy, ig, px[g], py[g], pz[g], valid[g], cell, ok);
#pragma unroll
            for (int j = 0; j < 4; ++j) slot[j] = valid[g][j] ? atomicAdd(&cur[cell[j] >> plan.bc_log2], 1u) : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (valid[g][j] && PI_BOUNDS(ctrl, slot[j], n, CS_SCATTER_REC))
                    rec[slot[j]] = make_float4(px[g][j], py[g][j], pz[g][j], __uint_as_float(ig + j));
        }
    }
}

// The cell of a bucket record (its system from the input index) and the
// system's constants.
__device__ __forceinline__ uint32_t record_cell(const Systems& sy, const float4& r, const SysDesc*& d)
{
    d = &sy.sys[system_of_particle(sy, __float_as_uint(r.w))];
    bool in = true;
    return cell_of(r.x, r.y, r.z, d->g, in) + d->cell_base;
}

// The sub-bin word of a cell with m members whose thermometers sum to
// (lo, hi) (see k_stabilise).
__device__ __forceinline__ uint2 xbin_word(uint32_t m, uint32_t lo, uint32_t hi)
{
    static_assert(XSUB == 8, "xbins packs 7 sub-bin starts and a flag into 8 bytes");
    return m > 255u ? make_uint2(0u, XBIN_COARSE << 24) : make_uint2(lo, hi | (m > DENSE_CELL ? XBIN_DENSE << 24 : 0u));
}

// Shared memory of k_bucket_cells.
struct CellSmem {
    float4 rec[BUCKET_CAP];        // the bucket's records in arrival order
    uint16_t cl[BUCKET_CAP];       // cell of record j, counted from the bucket's first cell
    uint16_t q[BUCKET_CAP];        // its place among its cell's records (arrival of the atomics)
    uint16_t idx[BUCKET_CAP];      // records in cell order: slot -> arrival index
    uint8_t sb[BUCKET_CAP];        // its x-sub-bin
    uint32_t cnt[BUCKET_MAX_CELLS];
    uint32_t start[BUCKET_MAX_CELLS + 1];
    uint32_t warp_sum[CELL_THREADS / 32];
    uint32_t warp_max[CELL_THREADS / 32];
};

__global__ void __launch_bounds__(CELL_THREADS) k_bucket_cells(
    const float4* __restrict__ rec, uint32_t n, Systems sy, BucketPlan plan, const uint32_t* __restrict__ base,
    uint32_t* __restrict__ counts, uint32_t* __restrict__ offsets, uint32_t* __restrict__ perm,
    float* __restrict__ sx, float* __restrict__ sy_out, float* __restrict__ sz, float4* __restrict__ P,
    uint2* __restrict__ xbins, float4* __restrict__ rec2, uint2* __restrict__ ovf_list, Ctrl* __restrict__ ctrl)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CellSmem& sm = *reinterpret_cast<CellSmem*>(smem_raw);
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t b = blockIdx.x;
    const uint32_t c0 = b << plan.bc_log2, c1 = min(c0 + (1u << plan.bc_log2), plan.C), ncell = c1 - c0;
    const uint32_t r0 = base[(size_t)b * plan.chunks], r1 = base[(size_t)(b + 1) * plan.chunks];
    const uint32_t M = r1 - r0;
    const bool big = M > (uint32_t)BUCKET_CAP;
    const uint32_t rows = __ldg(sy.rbase + sy.S);
    for (uint32_t c = tid; c < ncell; c += CELL_THREADS) sm.cnt[c] = 0u;
    __syncthreads();

    // count the cells (and keep the records of a bucket that fits); the
    // loads of a thread's records are all in flight before the first atomic
    bool bad = false;
    constexpr int PERT = BUCKET_CAP / CELL_THREADS;
    for (uint32_t j0 = tid; j0 < M; j0 += CELL_THREADS * PERT) {
        float4 r[PERT];
#pragma unroll
        for (int k = 0; k < PERT; ++k) {
            const uint32_t j = j0 + (uint32_t)k * CELL_THREADS;
            r[k] = j < M ? rec[r0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < PERT; ++k) {
            const uint32_t j = j0 + (uint32_t)k * CELL_THREADS;
            if (j >= M) continue;
            const SysDesc* d;
            const uint32_t c = record_cell(sy, r[k], d);
            if (c < c0 || c >= c1) { bad = true; continue; }
            const uint32_t q = atomicAdd(&sm.cnt[c - c0], 1u);
            if (!big) {
                sm.rec[j] = r[k];
                sm.cl[j] = (uint16_t)(c - c0);
                sm.q[j] = (uint16_t)q;
                sm.sb[j] = (uint8_t)x_sub_bin(r[k].x, c - d->cell_base, d->g);
            }
        }
    }
    if (bad) atomicOr(&ctrl->error, ERR_CAPACITY);
    __syncthreads();

    // exclusive scan of the cell counts (CELL_THREADS threads, up to four
    // cells each) and their maximum
    constexpr uint32_t PER = BUCKET_MAX_CELLS / CELL_THREADS;
    uint32_t v[PER], run = 0, mx = 0;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        const uint32_t c = tid * PER + k;
        v[k] = c < ncell ? sm.cnt[c] : 0u;
        mx = max(mx, v[k]);
        const uint32_t t = v[k];
        v[k] = run;
        run += t;
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 31) sm.warp_sum[warp] = incl;
    if (lane == 0) sm.warp_max[warp] = mx;
    __syncthreads();
    uint32_t before = 0, bmax = 0;
#pragma unroll
    for (int w = 0; w < CELL_THREADS / 32; ++w) {
        if (w < (int)warp) before += sm.warp_sum[w];
        bmax = max(bmax, sm.warp_max[w]);
    }
    const uint32_t excl = before + incl - run;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        const uint32_t c = tid * PER + k;
        if (c < ncell) sm.start[c] = excl + v[k];
    }
    if (tid == 0) {
        sm.start[ncell] = M;
        if (bmax) atomicMax(&ctrl->max_per_cell, bmax);
    }
    __syncthreads();

    // per cell: counts, offsets (Fig. 1), the sub-bin word of an empty
    // cell, and the sentinel slots of P after the last cell of an X-row
    for (uint32_t cl = tid; cl < ncell; cl += CELL_THREADS) {
        const uint32_t c = c0 + cl, m = sm.cnt[cl], at = r0 + sm.start[cl];
        counts[c] = m;
        offsets[c] = at;
        if (m == 0) xbins[c] = make_uint2(0u, 0u);
        const int sid = sy.S == 1 ? 0 : find_system(sy.cbase, sy.S, c);
        const SysDesc& d = sy.sys[sid];
        const uint32_t local = c - d.cell_base, nx = (uint32_t)d.g.n[0];
        if (local % nx == nx - 1u) {
            const uint32_t row = d.row_base + local / nx;
            const uint32_t pos = at + m + ROW_PADS * row;
            if (PI_BOUNDS(ctrl, pos + ROW_PADS - 1u, (uint64_t)n + ROW_PADS * (uint64_t)rows, CS_STAB_OUT)) {
#pragma unroll
                for (int k = 0; k < ROW_PADS; ++k)
                    P[pos + k] = make_float4(1e18f, 1e18f, 1e18f, __uint_as_float(0xffffffffu));
            }
        }
    }
    if (b == plan.B - 1u && tid == 0) offsets[plan.C] = n;

    if (big) {
        // the records in cell order for k_bucket_big (which ranks them);
        // the counts are re-used as cursors
        __syncthreads();
        for (uint32_t c = tid; c < ncell; c += CELL_THREADS) sm.cnt[c] = 0u;
        __syncthreads();
        for (uint32_t j = tid; j < M; j += CELL_THREADS) {
            const float4 r = rec[r0 + j];
            const SysDesc* d;
            const uint32_t c = record_cell(sy, r, d);
            if (c < c0 || c >= c1) continue;
            const uint32_t slot = sm.start[c - c0] + atomicAdd(&sm.cnt[c - c0], 1u);
            rec2[r0 + slot] = r;
        }
        if (tid == 0) {
            const unsigned long long old = atomicAdd(&ctrl->ovf, (1ull << 40) | (unsigned long long)M);
            const uint32_t e = (uint32_t)(old >> 40);
            if (PI_BOUNDS(ctrl, e, BUCKET_MAX, CS_STAB_OUT)) ovf_list[e] = make_uint2(b, (uint32_t)(old & OVF_MASK));
        }
        return;
    }

    // the records in cell order (arrival index by slot)
    for (uint32_t j = tid; j < M; j += CELL_THREADS) sm.idx[sm.start[sm.cl[j]] + sm.q[j]] = (uint16_t)j;
    __syncthreads();

    // per non-empty cell: the sub-bin word, the sum of its members'
    // thermometers
    for (uint32_t cl = tid; cl < ncell; cl += CELL_THREADS) {
        const uint32_t m0 = sm.start[cl], m1 = m0 + sm.cnt[cl];
        if (m1 == m0) continue;
        uint32_t lt_lo = 0, lt_hi = 0;
        for (uint32_t m = m0; m < m1; ++m) {
            const uint2 t = thermometer(sm.sb[sm.idx[m]]);
            lt_lo += t.x;
            lt_hi += t.y;
        }
        xbins[c0 + cl] = xbin_word(m1 - m0, lt_lo, lt_hi);
    }

    // per particle: stable rank and x-rank among its cell's members
    for (uint32_t s = tid; s < M; s += CELL_THREADS) {
        const uint32_t j = sm.idx[s];
        const float4 me = sm.rec[j];
        const uint32_t i = __float_as_uint(me.w), cl = sm.cl[j];
        const uint32_t m0 = sm.start[cl], m1 = m0 + sm.cnt[cl];
        uint32_t r = 0, xr = 0;
        for (uint32_t m = m0; m < m1; ++m) {
            const float4 o = sm.rec[sm.idx[m]];
            const uint32_t im = __float_as_uint(o.w);
            r += (im < i) ? 1u : 0u;
            xr += (o.x < me.x || (o.x == me.x && im < i)) ? 1u : 0u;
        }
        const uint32_t dst = r0 + m0 + r;
        if (!PI_BOUNDS(ctrl, dst, n, CS_STAB_OUT)) continue;
        perm[dst] = i;
        sx[dst] = me.x;
        sy_out[dst] = me.y;
        sz[dst] = me.z;
        const uint32_t c = c0 + cl;
        const int sid = sy.S == 1 ? 0 : find_system(sy.cbase, sy.S, c);
        const SysDesc& d = sy.sys[sid];
        const uint32_t row = d.row_base + (c - d.cell_base) / (uint32_t)d.g.n[0];
        const uint32_t at = r0 + m0 + xr + ROW_PADS * row;
        if (PI_BOUNDS(ctrl, at, (uint64_t)n + ROW_PADS * (uint64_t)rows, CS_STAB_OUT))
            P[at] = make_float4(me.x, me.y, me.z, __uint_as_float(dst));
    }
}

// The particles of the buckets k_bucket_cells left in cell order in rec2:
// one thread per particle, its cell's members read from rec2.
__global__ void __launch_bounds__(256) k_bucket_big(const float4* __restrict__ rec2, uint32_t n, Systems sy,
                                                    BucketPlan plan, const uint32_t* __restrict__ offsets,
                                                    uint32_t* __restrict__ perm, float* __restrict__ sx,
                                                    float* __restrict__ sy_out, float* __restrict__ sz,
                                                    float4* __restrict__ P, uint2* __restrict__ xbins,
                                                    const uint2* __restrict__ ovf_list, Ctrl* __restrict__ ctrl)
{
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    const unsigned long long o = *((volatile const unsigned long long*)&ctrl->ovf);
    const int nb = (int)min((unsigned long long)BUCKET_MAX, o >> 40);
    const uint32_t total = (uint32_t)(o & OVF_MASK);
    if (nb == 0) return;
    const uint32_t rows = __ldg(sy.rbase + sy.S);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        // the bucket of flattened overflow index t (list entries in order of
        // their first index)
        int lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ovf_list[mid].y <= t) lo = mid;
            else hi = mid - 1;
        }
        const uint2 e = ovf_list[lo];
        const uint32_t r0 = offsets[e.x << plan.bc_log2];
        const uint32_t k = r0 + (t - e.y);
        if (!PI_BOUNDS(ctrl, k, n, CS_STAB_MEMBER)) continue;
        const float4 me = rec2[k];
        const SysDesc* d;
        const uint32_t c = record_cell(sy, me, d);
        const uint32_t i = __float_as_uint(me.w);
        const uint32_t m0 = offsets[c], m1 = offsets[c + 1];
        if (!PI_BOUNDS(ctrl, m1, n + 1u, CS_STAB_MEMBER)) continue;
        uint32_t r = 0, xr = 0, lt_lo = 0, lt_hi = 0;
        for (uint32_t m = m0; m < m1; ++m) {
            const float4 q = rec2[m];
            const uint32_t im = __float_as_uint(q.w);
            r += (im < i) ? 1u : 0u;
            xr += (q.x < me.x || (q.x == me.x && im < i)) ? 1u : 0u;
            const uint2 th = thermometer(x_sub_bin(q.x, c - d->cell_base, d->g));
            lt_lo += th.x;
            lt_hi += th.y;
        }
        const uint32_t dst = m0 + r;
        perm[dst] = i;
        sx[dst] = me.x;
        sy_out[dst] = me.y;
        sz[dst] = me.z;
        const uint32_t row = d->row_base + (c - d->cell_base) / (uint32_t)d->g.n[0];
        const uint32_t at = m0 + xr + ROW_PADS * row;
        if (PI_BOUNDS(ctrl, at, (uint64_t)n + ROW_PADS * (uint64_t)rows, CS_STAB_OUT))
            P[at] = make_float4(me.x, me.y, me.z, __uint_as_float(dst));
        if (xr == 0) xbins[c] = xbin_word(m1 - m0, lt_lo, lt_hi);
    }
}

}  // namespace

bool bucket_plan(uint64_t n, uint64_t C, uint64_t mat_capacity, BucketPlan& plan)
{
    if (n == 0 || C == 0 || n >= (1ull << 31)) return false;
    // about 1024 particles per bucket on average: half of what a CTA ranks
    // in shared memory, so that uniform layouts (spread a few per cent)
    // never overflow
    const double q = (double)n / (double)C;
    uint32_t lg = 5;
    while (lg < 10 && (double)(1u << lg) * q < 1024.0) ++lg;
    while (lg <= 10 && ((C + (1ull << lg) - 1) >> lg) > (uint64_t)BUCKET_MAX) ++lg;
    if (lg > 10) return false;
    const uint64_t B = (C + (1ull << lg) - 1) >> lg;
    // buckets that would mostly overflow the shared-memory ranking take
    // the per-particle path instead
    if (n > B * (uint64_t)(BUCKET_CAP / 2)) return false;
    // chunks of BUCKET_CHUNK particles, fewer (and longer) if the count
    // matrix would not fit its buffer
    uint64_t chunks = (n + BUCKET_CHUNK - 1) / BUCKET_CHUNK;
    if (B * chunks + 1 > mat_capacity) chunks = (mat_capacity - 1) / B;
    if (chunks < 1) return false;
    plan.bc_log2 = lg;
    plan.B = (uint32_t)B;
    plan.chunks = (uint32_t)chunks;
    plan.C = (uint32_t)C;
    return true;
}

static uint32_t chunk_of(uint32_t n, const BucketPlan& plan)
{
    // particles per chunk, a multiple of 4 (the kernels load groups of 4)
    const uint64_t c = ((uint64_t)n + plan.chunks - 1) / plan.chunks;
    return (uint32_t)((c + 3) / 4 * 4);
}

cudaError_t launch_bucket_count(const float* x, const float* y, const float* z, uint32_t n, const Systems& sy,
                                const BucketPlan& plan, uint32_t* mat, Ctrl* ctrl, cudaStream_t s)
{
    const int vec = ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)z)) & 15u) == 0;
    return launch_dependent(k_bucket_count, dim3(plan.chunks), dim3(CHUNK_THREADS), (size_t)plan.B * 4u, s, x, y, z,
                            n, sy, plan, chunk_of(n, plan), mat, ctrl, vec);
}

cudaError_t launch_bucket_scatter(const float* x, const float* y, const float* z, uint32_t n,
                                  const Systems& sy, const BucketPlan& plan, const uint32_t* base, float4* rec,
                                  Ctrl* ctrl, cudaStream_t s)
{
    const int vec = ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)z)) & 15u) == 0;
    return launch_dependent(k_bucket_scatter, dim3(plan.chunks), dim3(CHUNK_THREADS), (size_t)plan.B * 4u, s, x, y,
                            z, n, sy, plan, chunk_of(n, plan), base, rec, ctrl, vec);
}

cudaError_t launch_bucket_cells(const float4* rec, uint32_t n, const Systems& sy, const BucketPlan& plan,
                                const uint32_t* base, uint32_t* counts, uint32_t* offsets, uint32_t* perm,
                                float* sx, float* sy_out, float* sz, float4* P, uint2* xbins, float4* rec2,
                                uint2* ovf_list, Ctrl* ctrl, cudaStream_t s)
{
    static_assert(BUCKET_CAP <= 65536 && BUCKET_MAX_CELLS <= 65536, "16-bit indices in shared memory");
    static_assert(BUCKET_MAX_CELLS % CELL_THREADS == 0, "the cell scan takes whole groups per thread");
    const size_t smem = sizeof(CellSmem);
    // the shared memory above the 48 KB default, allowed once per device
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static bool allowed[MAXDEV] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= MAXDEV || !allowed[dev]) {
            e = cudaFuncSetAttribute(k_bucket_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            if (dev >= 0 && dev < MAXDEV) allowed[dev] = true;
        }
    }
    return launch_dependent(k_bucket_cells, dim3(plan.B), dim3(CELL_THREADS), smem, s, rec, n, sy, plan, base,
                            counts, offsets, perm, sx, sy_out, sz, P, xbins, rec2, ovf_list, ctrl);
}

cudaError_t launch_bucket_big(const float4* rec2, uint32_t n, const Systems& sy, const BucketPlan& plan,
                              const uint32_t* offsets, uint32_t* perm, float* sx, float* sy_out, float* sz,
                              float4* P, uint2* xbins, const uint2* ovf_list, Ctrl* ctrl, int num_sms,
                              cudaStream_t s)
{
    // one wave: the kernel returns at once when no bucket overflowed
    return launch_dependent(k_bucket_big, dim3((unsigned)num_sms), dim3(256), 0, s, rec2, n, sy, plan, offsets,
                            perm, sx, sy_out, sz, P, xbins, ovf_list, ctrl);
}

}  // namespace pi
