// pi_radix.cu -- binning (a1-a4 of Sec. 2) as a stable radix sort of the
// particles by cell.
//
// The same results as the per-particle path of pi_bin.cu (counts, offsets,
// M_C, the stable permutation, the sorted SoA, the row-padded x-ordered copy
// P and each cell's sub-bin starts, bit for bit):
//
//   k_radix_keys     per chunk of 4096 input particles: the global cell of
//                    each (the key) and a histogram of its first digit,
//                    written as one column of the digit x chunk matrix
//   k_scan           (pi_bin.cu) exclusive scan of that matrix in digit-major
//                    order: where each chunk's keys of each digit go
//   k_radix_scatter  per chunk, a stable split by the digit: each warp ranks
//                    its 256 consecutive keys in order (warp matches and
//                    running per-digit counters), the warps' counts are
//                    scanned per digit, and every key and its input index go
//                    to their place -- a least-significant-digit radix pass
//   k_radix_count    per chunk, the histogram of the next digit of the keys
//                    the last pass wrote (then k_scan and the next scatter)
//   k_radix_gather   per sorted slot: perm, the sorted positions (gathered
//                    by input index), and the offsets of Fig. 1 from the
//                    sorted keys (a cell starts where the key first reaches
//                    it)
//   k_radix_rank     per cell: count, M_C, an empty cell's sub-bin word and
//                    P's row pads; per slot: the x-rank among the cell's
//                    members (ties by input index) and its P record, and
//                    for x-rank 0 the cell's sub-bin word
// Least-significant-digit passes are stable and the first pass reads the
// particles in input order, so inside a cell the keys end in input order:
// the stable rank of Sec. 2's scatter without a per-cell ranking.
#include <algorithm>

#include "pi_internal.cuh"

namespace pi {

namespace {

constexpr int RADIX_THREADS = 512;                 // 16 warps
constexpr int RADIX_WARPS = RADIX_THREADS / 32;
constexpr int RADIX_PER_WARP = RADIX_CHUNK / RADIX_WARPS;  // 256 keys, 8 rounds of 32
constexpr int RADIX_ROUNDS = RADIX_PER_WARP / 32;
constexpr unsigned FULL_MASK = 0xffffffffu;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__global__ void __launch_bounds__(RADIX_THREADS) k_radix_keys(const float* __restrict__ x,
                                                              const float* __restrict__ y,
                                                              const float* __restrict__ z, uint32_t n,
                                                              Systems sy, RadixPlan plan,
                                                              uint32_t* __restrict__ keys,
                                                              uint32_t* __restrict__ mat, Ctrl* __restrict__ ctrl,
                                                              int vec)
{
    extern __shared__ uint32_t hist[];
    pdl_trigger();
    for (uint32_t b = threadIdx.x; b < plan.bins; b += RADIX_THREADS) hist[b] = 0u;
    __syncthreads();
    pdl_wait();  // the particle bases and the control block are k_zero's
    const uint32_t k = blockIdx.x;
    const uint32_t beg = k * RADIX_CHUNK, end = min(beg + RADIX_CHUNK, n);
    const uint32_t mask = plan.bins - 1u;
    bool ok = true;
    for (uint32_t i0 = beg + 4u * threadIdx.x; i0 < end; i0 += 4u * RADIX_THREADS) {
        float px[4], py[4], pz[4];
        bool valid[4];
        uint32_t cell[4];
        load4(x, y, z, i0, end, vec, px, py, pz, valid);
        cells4(sy, i0, px, py, pz, valid, cell, ok);
        if (vec && i0 + 4u <= end) {
            *reinterpret_cast<uint4*>(keys + i0) = make_uint4(cell[0], cell[1], cell[2], cell[3]);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (valid[j]) keys[i0 + j] = cell[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (valid[j]) atomicAdd(&hist[cell[j] & mask], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < plan.bins; b += RADIX_THREADS) mat[(size_t)b * plan.chunks + k] = hist[b];
    if (!ok) atomicOr(&ctrl->error, ERR_OUT_OF_BOX);
}

// Histogram of the digit at `shift` of a chunk of keys.
__global__ void __launch_bounds__(RADIX_THREADS) k_radix_count(const uint32_t* __restrict__ keys, uint32_t n,
                                                               RadixPlan plan, uint32_t shift,
                                                               uint32_t* __restrict__ mat, Ctrl* __restrict__ ctrl)
{
    extern __shared__ uint32_t hist[];
    pdl_trigger();
    for (uint32_t b = threadIdx.x; b < plan.bins; b += RADIX_THREADS) hist[b] = 0u;
    __syncthreads();
    pdl_wait();
    if (cta_error(ctrl)) return;
    const uint32_t k = blockIdx.x;
    const uint32_t beg = k * RADIX_CHUNK, end = min(beg + RADIX_CHUNK, n);
    const uint32_t mask = plan.bins - 1u;
    for (uint32_t i = beg + threadIdx.x; i < end; i += RADIX_THREADS) atomicAdd(&hist[(keys[i] >> shift) & mask], 1u);
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < plan.bins; b += RADIX_THREADS) mat[(size_t)b * plan.chunks + k] = hist[b];
}

// One stable pass by the digit at `shift`.  vals_in = nullptr: the values
// are the input positions (the first pass).  Shared memory: the warps'
// running counters [RADIX_WARPS][bins] and the chunk's global digit bases
// [bins].
__global__ void __launch_bounds__(RADIX_THREADS) k_radix_scatter(const uint32_t* __restrict__ keys_in,
                                                                 const uint32_t* __restrict__ vals_in,
                                                                 uint32_t* __restrict__ keys_out,
                                                                 uint32_t* __restrict__ vals_out, uint32_t n,
                                                                 RadixPlan plan, uint32_t shift,
                                                                 const uint32_t* __restrict__ base,
                                                                 Ctrl* __restrict__ ctrl)
{
    extern __shared__ uint32_t sm[];
    const uint32_t bins = plan.bins, mask = bins - 1u;
    uint32_t* cnt = sm;                           // [warp][bins]
    uint32_t* gb = sm + RADIX_WARPS * bins;       // [bins]
    pdl_trigger();
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t b = lane; b < bins; b += 32) cnt[warp * bins + b] = 0u;
    pdl_wait();
    if (cta_error(ctrl)) return;
    const uint32_t k = blockIdx.x;
    for (uint32_t b = threadIdx.x; b < bins; b += RADIX_THREADS) gb[b] = base[(size_t)b * plan.chunks + k];
    __syncwarp();
    // the warp's keys in order, 32 per round: each key's place among the
    // warp's keys of its digit so far
    const uint32_t w0 = k * RADIX_CHUNK + warp * RADIX_PER_WARP;
    const unsigned lt = lanemask_lt();
    uint32_t kk[RADIX_ROUNDS], vv[RADIX_ROUNDS], loc[RADIX_ROUNDS];
#pragma unroll
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        const uint32_t q = w0 + (uint32_t)r * 32u + lane;
        const bool valid = q < n;
        kk[r] = valid ? keys_in[q] : 0u;
        vv[r] = valid ? (vals_in ? vals_in[q] : q) : 0u;
    }
#pragma unroll
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        const uint32_t q = w0 + (uint32_t)r * 32u + lane;
        const bool valid = q < n;
        const uint32_t d = (kk[r] >> shift) & mask;
        const unsigned peers = __match_any_sync(FULL_MASK, valid ? d : 0xffffffffu);
        const uint32_t before = cnt[warp * bins + (valid ? d : 0u)];
        __syncwarp();
        if (valid && (peers & lt) == 0u) cnt[warp * bins + d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        loc[r] = before + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive scan over the warps (warp order = key order)
    for (uint32_t b = threadIdx.x; b < bins; b += RADIX_THREADS) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RADIX_WARPS; ++w) {
            const uint32_t t = cnt[w * bins + b];
            cnt[w * bins + b] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        const uint32_t q = w0 + (uint32_t)r * 32u + lane;
        if (q >= n) continue;
        const uint32_t d = (kk[r] >> shift) & mask;
        const uint32_t pos = gb[d] + cnt[warp * bins + d] + loc[r];
        if (!PI_BOUNDS(ctrl, pos, n, CS_SCATTER_REC)) continue;
        keys_out[pos] = kk[r];
        vals_out[pos] = vv[r];
    }
}

// Per sorted slot: perm, sorted positions, and the offsets of the cells
// from the previous slot's cell (exclusive) to its own (inclusive); the
// last slot also ends the cells after it.
__global__ void __launch_bounds__(256) k_radix_gather(const uint32_t* __restrict__ keys,
                                                      const uint32_t* __restrict__ vals,
                                                      const float* __restrict__ x, const float* __restrict__ y,
                                                      const float* __restrict__ z, uint32_t n, uint32_t C,
                                                      uint32_t* __restrict__ offsets, uint32_t* __restrict__ perm,
                                                      float* __restrict__ sx, float* __restrict__ sy_out,
                                                      float* __restrict__ sz, Ctrl* __restrict__ ctrl)
{
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    bool bad = false;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t c = keys[k], i = vals[k];
        const uint32_t c0 = k == 0 ? 0u : keys[k - 1] + 1u;
        if (c >= C || i >= n) { bad = true; continue; }
        for (uint32_t cc = c0; cc <= c; ++cc) offsets[cc] = k;
        if (k == n - 1u)
            for (uint32_t cc = c + 1u; cc <= C; ++cc) offsets[cc] = n;
        perm[k] = i;
        sx[k] = x[i];
        sy_out[k] = y[i];
        sz[k] = z[i];
    }
    if (bad) atomicOr(&ctrl->error, ERR_CAPACITY);
}

// Per cell (t < C) and per sorted slot (t < n), grid-stride over both.
__global__ void __launch_bounds__(256) k_radix_rank(const uint32_t* __restrict__ keys, uint32_t n, Systems sy,
                                                    uint32_t C, const uint32_t* __restrict__ offsets,
                                                    const uint32_t* __restrict__ perm,
                                                    const float* __restrict__ sx, const float* __restrict__ sy_in,
                                                    const float* __restrict__ sz, uint32_t* __restrict__ counts,
                                                    float4* __restrict__ P, uint2* __restrict__ xbins,
                                                    Ctrl* __restrict__ ctrl)
{
    pdl_trigger();
    pdl_wait();
    if (cta_error(ctrl)) return;
    const uint32_t rows = __ldg(sy.rbase + sy.S);
    const uint64_t np = (uint64_t)n + ROW_PADS * (uint64_t)rows;
    uint32_t mx = 0;
    bool bad = false;
    const uint32_t total = max(n, C);
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        if (t < C) {
            const uint32_t o0 = offsets[t], o1 = offsets[t + 1], m = o1 - o0;
            const bool cell_ok = o0 <= o1 && o1 <= n;
            bad |= !cell_ok;
            counts[t] = m;
            mx = max(mx, m);
            if (m == 0) xbins[t] = make_uint2(0u, 0u);
            const int sid = sy.S == 1 ? 0 : find_system(sy.cbase, sy.S, t);
            const SysDesc& d = sy.sys[sid];
            const uint32_t local = t - d.cell_base, nx = (uint32_t)d.g.n[0];
            if (cell_ok && local % nx == nx - 1u) {
                const uint32_t pos = o1 + ROW_PADS * (d.row_base + local / nx);
                if (PI_BOUNDS(ctrl, pos + ROW_PADS - 1u, np, CS_STAB_OUT)) {
#pragma unroll
                    for (int k = 0; k < ROW_PADS; ++k)
                        P[pos + k] = make_float4(1e18f, 1e18f, 1e18f, __uint_as_float(0xffffffffu));
                }
            }
        }
        if (t < n) {
            const uint32_t c = keys[t];
            if (c >= C) { bad = true; continue; }
            const uint32_t m0 = offsets[c], m1 = offsets[c + 1];
            if (m0 > t || t >= m1 || m1 > n) { bad = true; continue; }
            const float xm = sx[t];
            const uint32_t im = perm[t];
            const int sid = sy.S == 1 ? 0 : find_system(sy.cbase, sy.S, c);
            const SysDesc& d = sy.sys[sid];
            uint32_t xr = 0;
            for (uint32_t q = m0; q < m1; ++q) {
                const float xq = sx[q];
                xr += (xq < xm || (xq == xm && perm[q] < im)) ? 1u : 0u;
            }
            const uint32_t row = d.row_base + (c - d.cell_base) / (uint32_t)d.g.n[0];
            const uint64_t at = (uint64_t)m0 + xr + ROW_PADS * (uint64_t)row;
            if (PI_BOUNDS(ctrl, at, np, CS_STAB_OUT)) P[at] = make_float4(xm, sy_in[t], sz[t], __uint_as_float(t));
            if (xr == 0) {
                // the cell's sub-bin word: the sum of its members' thermometers
                uint32_t lo = 0, hi = 0;
                for (uint32_t q = m0; q < m1; ++q) {
                    const uint2 th = thermometer(x_sub_bin(sx[q], c - d.cell_base, d.g));
                    lo += th.x;
                    hi += th.y;
                }
                const uint32_t m = m1 - m0;
                xbins[c] = m > 255u ? make_uint2(0u, XBIN_COARSE << 24)
                                    : make_uint2(lo, hi | (m > DENSE_CELL ? XBIN_DENSE << 24 : 0u));
            }
        }
    }
    // M_C: each warp's maximum, one atomic per warp
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
    if ((threadIdx.x & 31u) == 0u && mx) atomicMax(&ctrl->max_per_cell, mx);
    if (bad) atomicOr(&ctrl->error, ERR_CAPACITY);
}

}  // namespace

bool radix_plan(uint64_t n, uint64_t C, uint64_t mat_capacity, RadixPlan& plan)
{
    if (n == 0 || C == 0 || n >= (1ull << 31) || C >= (1ull << 31)) return false;
    uint32_t bits = 1;
    while ((1ull << bits) < C) ++bits;
    const uint32_t passes = (bits + RADIX_MAX_BITS - 1) / RADIX_MAX_BITS;
    const uint32_t digit = (bits + passes - 1) / passes;
    const uint64_t chunks = (n + RADIX_CHUNK - 1) / RADIX_CHUNK;
    if (((uint64_t)1 << digit) * chunks + 1 > mat_capacity) return false;
    plan.passes = passes;
    plan.digit_bits = digit;
    plan.bins = 1u << digit;
    plan.chunks = (uint32_t)chunks;
    plan.C = (uint32_t)C;
    return true;
}

cudaError_t launch_radix_keys(const float* x, const float* y, const float* z, uint32_t n, const Systems& sy,
                              const RadixPlan& plan, uint32_t* keys, uint32_t* mat, Ctrl* ctrl, cudaStream_t s)
{
    const int vec = ((((uintptr_t)x) | ((uintptr_t)y) | ((uintptr_t)z) | ((uintptr_t)keys)) & 15u) == 0;
    return launch_dependent(k_radix_keys, dim3(plan.chunks), dim3(RADIX_THREADS), (size_t)plan.bins * 4u, s, x, y, z,
                            n, sy, plan, keys, mat, ctrl, vec);
}

cudaError_t launch_radix_count(const uint32_t* keys, uint32_t n, const RadixPlan& plan, uint32_t shift,
                               uint32_t* mat, Ctrl* ctrl, cudaStream_t s)
{
    return launch_dependent(k_radix_count, dim3(plan.chunks), dim3(RADIX_THREADS), (size_t)plan.bins * 4u, s, keys, n,
                            plan, shift, mat, ctrl);
}

cudaError_t launch_radix_scatter(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                                 uint32_t* vals_out, uint32_t n, const RadixPlan& plan, uint32_t shift,
                                 const uint32_t* base, Ctrl* ctrl, cudaStream_t s)
{
    const size_t smem = (size_t)(RADIX_WARPS + 1) * plan.bins * 4u;  // at most 17 x 512 words
    return launch_dependent(k_radix_scatter, dim3(plan.chunks), dim3(RADIX_THREADS), smem, s, keys_in, vals_in,
                            keys_out, vals_out, n, plan, shift, base, ctrl);
}

cudaError_t launch_radix_gather(const uint32_t* keys, const uint32_t* vals, const float* x, const float* y,
                                const float* z, uint32_t n, uint32_t C, uint32_t* offsets, uint32_t* perm, float* sx,
                                float* sy_out, float* sz, Ctrl* ctrl, int num_sms, cudaStream_t s)
{
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((n + 255) / 256, (uint32_t)num_sms * 8u));
    return launch_dependent(k_radix_gather, dim3(blocks), dim3(256), 0, s, keys, vals, x, y, z, n, C, offsets, perm,
                            sx, sy_out, sz, ctrl);
}

cudaError_t launch_radix_rank(const uint32_t* keys, uint32_t n, const Systems& sy, uint32_t C,
                              const uint32_t* offsets, const uint32_t* perm, const float* sx, const float* sy_in,
                              const float* sz, uint32_t* counts, float4* P, uint2* xbins, Ctrl* ctrl, int num_sms,
                              cudaStream_t s)
{
    const uint32_t total = std::max(n, C);
    const uint32_t blocks = std::max<uint32_t>(1, std::min<uint32_t>((total + 255) / 256, (uint32_t)num_sms * 8u));
    return launch_dependent(k_radix_rank, dim3(blocks), dim3(256), 0, s, keys, n, sy, C, offsets, perm, sx, sy_in, sz,
                            counts, P, xbins, ctrl);
}

}  // namespace pi
