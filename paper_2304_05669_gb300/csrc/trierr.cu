// Per-triangle rendering error (Sec. 4.4): rendering without the emission
// term leaves large error exactly where the emitters are.  Pixels are
// grouped by their first-hit triangle with a stable radix sort, each
// triangle's segment boundaries are marked in one pass over the sorted
// keys, and one warp per triangle sums its pixels' squared errors in FP64
// (lane l takes pixels l, l + 32, ... of the segment in order, then a fixed
// butterfly), so the result is deterministic.
#include "fipt_internal.cuh"

namespace {

__global__ void k_tri_keys(const int32_t* __restrict__ tri, int64_t stride, int64_t P, int64_t T,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int32_t t = tri[p * stride];
    keys[p] = (t >= 0 && t < T) ? (uint32_t)t : (uint32_t)T;   // T = "no triangle", sorts last
    vals[p] = (uint32_t)p;
}

__global__ void k_mark_segments(const uint32_t* __restrict__ keys, int64_t P, int64_t T,
                                int32_t* __restrict__ seg_begin, int32_t* __restrict__ seg_end) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= P) return;
    const uint32_t k = keys[j];
    if (k >= (uint32_t)T) return;
    if (j == 0 || keys[j - 1] != k) seg_begin[k] = (int32_t)j;
    if (j == P - 1 || keys[j + 1] != k) seg_end[k] = (int32_t)(j + 1);
}

__global__ void k_segment_sums(const uint32_t* __restrict__ pix, const int32_t* __restrict__ seg_begin,
                               const int32_t* __restrict__ seg_end, const float* __restrict__ Lr,
                               const float* __restrict__ Lgt, int64_t T, double* __restrict__ err,
                               int32_t* __restrict__ count) {
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= T) return;                      // whole warp
    const int32_t b = seg_begin[t], e = seg_end[t];
    double s = 0.0;
    for (int32_t j = b + lane; j < e; j += 32) {
        const int64_t p = pix[j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double d = (double)Lr[3 * p + c] - (double)Lgt[3 * p + c];
            s = fma(d, d, s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        err[t] = s;
        count[t] = e - b;
    }
}

struct TriErrLayout {
    uint32_t *keys, *keys_alt, *vals, *vals_alt, *hist;
    int32_t *seg_begin, *seg_end;
    size_t bytes;
};

TriErrLayout carve(void* ws, int64_t P, int64_t T) {
    Carver c{static_cast<char*>(ws), 0};
    TriErrLayout L;
    const int64_t p1 = P > 0 ? P : 1, t1 = T > 0 ? T : 1;
    L.keys = c.take<uint32_t>((size_t)p1);
    L.keys_alt = c.take<uint32_t>((size_t)p1);
    L.vals = c.take<uint32_t>((size_t)p1);
    L.vals_alt = c.take<uint32_t>((size_t)p1);
    L.hist = c.take<uint32_t>(radix_sort_scratch_bytes(p1) / sizeof(uint32_t));
    L.seg_begin = c.take<int32_t>((size_t)t1);
    L.seg_end = c.take<int32_t>((size_t)t1);
    L.bytes = c.off + 256;
    return L;
}

inline unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

extern "C" fipt_status fipt_tri_error_workspace_size(int64_t P, int64_t T, size_t* bytes) {
    FIPT_REQUIRE(bytes && P >= 0 && T >= 0 && P < ((int64_t)1 << 31) && T < ((int64_t)1 << 31) - 1,
                 "bad arguments");
    *bytes = carve(nullptr, P, T).bytes;
    return FIPT_OK;
}

extern "C" fipt_status fipt_tri_error(const int32_t* tri, int64_t tri_stride, const float* Lr,
                                      const float* Lgt, int64_t P, int64_t T, double* err_sum, int32_t* count, void* ws,
                                      size_t ws_bytes, fipt_stream stream) {
    FIPT_REQUIRE(P >= 0 && T >= 0 && P < ((int64_t)1 << 31) && T < ((int64_t)1 << 31) - 1,
                 "bad sizes P=%lld T=%lld", (long long)P, (long long)T);
    FIPT_REQUIRE(tri_stride >= 1, "tri_stride must be >= 1");
    if (T == 0) return FIPT_OK;
    FIPT_REQUIRE(err_sum && count && fipt_aligned(err_sum, 8) && fipt_aligned(count, 4),
                 "err_sum / count NULL or misaligned");
    FIPT_REQUIRE(P == 0 || (tri && Lr && Lgt && fipt_aligned(tri, 4) && fipt_aligned(Lr, 4) &&
                            fipt_aligned(Lgt, 4)), "tri / Lr / Lgt NULL or misaligned");
    TriErrLayout L = carve(ws, P, T);
    if (!ws || ws_bytes < L.bytes || !fipt_aligned(ws, 256))
        return fipt_set_error(FIPT_ERR_WORKSPACE, "tri_error workspace %zu < %zu bytes (256-aligned)",
                              ws_bytes, L.bytes);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    FIPT_CUDA(cudaMemsetAsync(L.seg_begin, 0, sizeof(int32_t) * (size_t)T, st));
    FIPT_CUDA(cudaMemsetAsync(L.seg_end, 0, sizeof(int32_t) * (size_t)T, st));
    uint32_t* sk = L.keys;
    uint32_t* sv = L.vals;
    if (P > 0) {
        FIPT_LAUNCH(k_tri_keys, blocks(P, 256), 256, 0, st, tri, tri_stride, P, T, L.keys, L.vals);
        int bits = 0;
        while (((int64_t)1 << bits) <= T) ++bits;      // keys lie in [0, T]
        bits = (bits + 7) & ~7;
        fipt_status r = radix_sort_pairs<uint32_t>(L.keys, L.keys_alt, L.vals, L.vals_alt, L.hist, P,
                                                   bits, st, &sk, &sv);
        if (r != FIPT_OK) return r;
        FIPT_LAUNCH(k_mark_segments, blocks(P, 256), 256, 0, st, sk, P, T, L.seg_begin, L.seg_end);
    }
    FIPT_LAUNCH(k_segment_sums, blocks(T * 32, 256), 256, 0, st, sv, L.seg_begin, L.seg_end, Lr, Lgt, T,
                err_sum, count);
    FIPT_LAUNCHED("tri_error");
    return FIPT_OK;
}
