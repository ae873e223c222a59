// Device primitives: exclusive scan and a stable LSD radix sort of
// (uint64 key, int32 value) pairs.  Used by the partition (faces and vertex
// copies ordered by piece, then by global id) and by the metrics (quantiles).
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "pgcp_internal.h"

namespace pgcp {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename TIn>
__global__ void k_scan_tiles(const TIn* __restrict__ in, int64_t* __restrict__ out, int64_t* __restrict__ tile_sums,
                             int64_t n) {
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t v[SCAN_ITEMS];
    int64_t acc = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        v[i] = (idx < n) ? (int64_t)in[idx] : 0;
        acc += v[i];
    }
    // inclusive scan of per-thread totals inside the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t t = (lane < SCAN_THREADS / 32) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t excl = x - acc + (warp > 0 ? warp_tot[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = excl;
        excl += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) tile_sums[blockIdx.x] = excl;
}

__global__ void k_scan_add(int64_t* __restrict__ out, const int64_t* __restrict__ tile_off, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int64_t add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

template <typename TIn>
void scan_impl(const TIn* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return;
    }
    int64_t nt = ceil_div(n, SCAN_TILE);
    DBuf<int64_t> sums;
    sums.alloc(nt + 1, s);
    { k_scan_tiles<TIn><<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, out, sums.p, n); ::pgcp::note_launch(); }
    PGCP_CUDA(cudaGetLastError());
    if (nt > 1) {
        DBuf<int64_t> offs;
        offs.alloc(nt + 1, s);
        scan_impl<int64_t>(sums.p, offs.p, nt, s, nullptr);
        { k_scan_add<<<(unsigned)nt, 256, 0, s>>>(out, offs.p, n); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        if (total_host) {
            int64_t a = 0, b = 0;
            PGCP_CUDA(cudaMemcpyAsync(&a, offs.p + nt - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaMemcpyAsync(&b, sums.p + nt - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
            PGCP_CUDA(cudaStreamSynchronize(s));
            *total_host = a + b;
        }
    } else if (total_host) {
        PGCP_CUDA(cudaMemcpyAsync(total_host, sums.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PGCP_CUDA(cudaStreamSynchronize(s));
    }
}

// ---------------------------------------------------------------- radix sort

constexpr int RS_THREADS = 256;
constexpr int RS_CHUNKS = 8;
constexpr int RS_TILE = RS_THREADS * RS_CHUNKS;

__global__ void k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift, int64_t nblocks,
                          int64_t* __restrict__ counts) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        int64_t idx = base + i;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                             uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t n, int shift,
                             int64_t nblocks, const int64_t* __restrict__ offs) {
    __shared__ int64_t tile_off[256];
    __shared__ int wcount[RS_THREADS / 32][256];
    __shared__ int ctot[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    tile_off[threadIdx.x] = offs[(int64_t)threadIdx.x * nblocks + blockIdx.x];
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int c = 0; c < RS_CHUNKS; ++c) {
        for (int w = 0; w < RS_THREADS / 32; ++w) wcount[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t idx = base + (int64_t)c * RS_THREADS + threadIdx.x;
        const bool valid = idx < n;
        uint64_t k = valid ? kin[idx] : 0;
        int32_t v = valid ? vin[idx] : 0;
        unsigned d = valid ? (unsigned)((k >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & ((1u << lane) - 1u));
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcount[warp][d] = __popc(peers);
        __syncthreads();
        {
            int s = 0;
            for (int w = 0; w < RS_THREADS / 32; ++w) {
                int t = wcount[w][threadIdx.x];
                wcount[w][threadIdx.x] = s;
                s += t;
            }
            ctot[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) {
            int64_t pos = tile_off[d] + wcount[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        tile_off[threadIdx.x] += ctot[threadIdx.x];
        __syncthreads();
    }
}

}  // namespace

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    scan_impl<int64_t>(in, out, n, s, total_host);
}

void exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s, int64_t* total_host) {
    scan_impl<int32_t>(in, out, n, s, total_host);
}

void radix_sort_pairs(uint64_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return;
    int64_t nb = ceil_div(n, RS_TILE);
    DBuf<uint64_t> k2;
    DBuf<int32_t> v2;
    DBuf<int64_t> counts, offs;
    k2.alloc(n, s);
    v2.alloc(n, s);
    counts.alloc(256 * nb, s);
    offs.alloc(256 * nb, s);
    uint64_t *ka = keys, *kb = k2.p;
    int32_t *va = vals, *vb = v2.p;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        { k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, s>>>(ka, n, shift, nb, counts.p); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        exclusive_scan_i64(counts.p, offs.p, 256 * nb, s, nullptr);
        { k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, nb, offs.p); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        PGCP_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        PGCP_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
}

// ---- variants on caller-provided workspace (no allocation)

int64_t sort_ws_counts(int64_t n) { return 256 * ceil_div(std::max<int64_t>(n, 1), RS_TILE); }

void scan_noalloc(const int64_t* in, int64_t* out, int64_t n, int64_t* ws, int64_t ws_len, cudaStream_t s) {
    // two levels: tile sums [nt], their scan [nt]; nt must fit one tile
    const int64_t nt = ceil_div(n, SCAN_TILE);
    if (nt > SCAN_TILE || 2 * (nt + 1) + 2 > ws_len) fail(PGCP_E_ARG, "scan workspace too small");
    int64_t* sums = ws;
    int64_t* offs = ws + nt + 1;
    int64_t* top = ws + 2 * (nt + 1);
    { k_scan_tiles<int64_t><<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, out, sums, n); ::pgcp::note_launch(); }
    if (nt > 1) {
        { k_scan_tiles<int64_t><<<1, SCAN_THREADS, 0, s>>>(sums, offs, top, nt); ::pgcp::note_launch(); }
        { k_scan_add<<<(unsigned)nt, 256, 0, s>>>(out, offs, n); ::pgcp::note_launch(); }
    }
    PGCP_CUDA(cudaGetLastError());
}

void radix_sort_pairs_noalloc(uint64_t* keys, int32_t* vals, int64_t n, int bits, cudaStream_t s, uint64_t* k2,
                              int32_t* v2, int64_t* counts, int64_t* offs, int64_t* scan_ws, int64_t scan_ws_len) {
    if (n <= 1 || bits <= 0) return;
    const int64_t nb = ceil_div(n, RS_TILE);
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        { k_rs_hist<<<(unsigned)nb, RS_THREADS, 0, s>>>(ka, n, shift, nb, counts); ::pgcp::note_launch(); }
        scan_noalloc(counts, offs, 256 * nb, scan_ws, scan_ws_len, s);
        { k_rs_scatter<<<(unsigned)nb, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, nb, offs); ::pgcp::note_launch(); }
        PGCP_CUDA(cudaGetLastError());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        PGCP_CUDA(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        PGCP_CUDA(cudaMemcpyAsync(vals, va, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
}

uint32_t read_errors(pgcp_ctx* ctx) {
    uint32_t e = 0;
    PGCP_CUDA(cudaMemcpyAsync(&e, ctx->err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    PGCP_CUDA(cudaStreamSynchronize(ctx->stream));
    return e;
}

}  // namespace pgcp
