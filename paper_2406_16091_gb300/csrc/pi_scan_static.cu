// pi_scan_static.cu -- the exclusive scan of per-cell counts (the a3 kernel,
// k_scan) for callers that cannot allocate device memory.
//
// The scan needs scratch: a control block (tile ticket, error bits, M_C) and
// one lookback descriptor per 4096-count tile.  pi_bin keeps that scratch in
// the arena pi_create allocates.  This entry point keeps it instead in one
// file-scope __device__ array of fixed size, so it calls no cudaMalloc, no
// cudaFree and no allocating library routine; the caller passes the counts
// and the output offsets.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code cannot use the array's name as a device address (it
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and caches
// it; later calls on that device reuse the cached address.
#include <cstdio>
#include <mutex>

#include "pi.h"
#include "pi_internal.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_CELLS = (int64_t)1 << 24;
constexpr size_t NOALLOC_TILES = (size_t)((NOALLOC_MAX_CELLS + 1 + pi::SCAN_TILE - 1) / pi::SCAN_TILE);
constexpr size_t NOALLOC_BYTES = sizeof(pi::Ctrl) + NOALLOC_TILES * sizeof(unsigned long long);
constexpr int NOALLOC_MAX_DEVICES = 64;

void* g_scratch_addr[NOALLOC_MAX_DEVICES];
cudaError_t g_setup_err[NOALLOC_MAX_DEVICES];
std::once_flag g_setup_once[NOALLOC_MAX_DEVICES];

}  // namespace

namespace pi {
void set_last_error_text(const char* text);
}

// Control block followed by the tile descriptors; shared by every call.
static __device__ __align__(256) unsigned char g_scan_scratch[NOALLOC_BYTES];

extern "C" pi_status pi_scan_counts_noalloc(const uint32_t* counts, int64_t C, uint32_t* offsets,
                                            uint32_t* result, pi_stream stream)
{
    if (!counts || !offsets || C < 1) return PI_ERR_INVALID_ARG;
    if (C > NOALLOC_MAX_CELLS) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "pi_scan_counts_noalloc: %lld cells exceed the fixed scratch limit of %lld",
                      (long long)C, (long long)NOALLOC_MAX_CELLS);
        pi::set_last_error_text(msg);
        return PI_ERR_CAPACITY;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PI_ERR_CUDA;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return PI_ERR_CAPACITY;
    // once per device, with that device current: the device address of the array
    std::call_once(g_setup_once[dev], [dev] {
        g_setup_err[dev] = cudaGetSymbolAddress(&g_scratch_addr[dev], g_scan_scratch);
    });
    if (g_setup_err[dev] != cudaSuccess || !g_scratch_addr[dev]) return PI_ERR_CUDA;

    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)g_scratch_addr[dev];
    pi::Ctrl* ctrl = (pi::Ctrl*)base;
    unsigned long long* status = (unsigned long long*)(base + sizeof(pi::Ctrl));
    const size_t tiles = (size_t)((C + 1 + pi::SCAN_TILE - 1) / pi::SCAN_TILE);
    // the array keeps the previous call's contents: clear the control block
    // and the descriptors this call uses (a cleared descriptor reads as "not
    // ready", so one fixed epoch suffices)
    const size_t words = (sizeof(pi::Ctrl) + tiles * sizeof(unsigned long long)) / 4;
    if (pi::launch_zero((uint32_t*)base, words, nullptr, nullptr, 0, s) != cudaSuccess) return PI_ERR_CUDA;
    if (pi::launch_scan(counts, (uint32_t)C, offsets, status, ctrl, 1u, 1000000000ull, 0, s) !=
        cudaSuccess)
        return PI_ERR_CUDA;
    if (result) {
        if (cudaMemcpyAsync(result, &ctrl->max_per_cell, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess ||
            cudaMemcpyAsync(result + 1, &ctrl->error, sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                            s) != cudaSuccess)
            return PI_ERR_CUDA;
    }
    return PI_OK;
}
