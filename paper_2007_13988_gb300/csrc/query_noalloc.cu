// pifu_query_noalloc: the occupancy query (pifu_query) for callers that
// cannot allocate device memory themselves -- for example code running
// inside a host application whose own allocator owns every byte of device
// memory, or in a plug-in/callback environment where calling cudaMalloc is
// not permitted.  Such a caller cannot create a context (pifu_create
// allocates the weights and a workspace), so this entry point needs none:
// the network comes from a device copy of the weight blob that the caller
// placed in memory it already owns, inputs and outputs are the caller's, and
// the MLP activations live in one fixed, file-scope device array.
//
// That array (kScratchBytes = 16 MiB) is part of the library's image: every
// GPU that loads the library holds it until the process exits.  All calls
// share it, so calls whose work overlaps on the GPU (different streams,
// threads or processes' streams on one context) race and must be
// serialised by the caller.  A call writes every scratch row before it
// reads it, so nothing in the array has to start at zero and the previous
// call's leftovers are never read.  The array bounds the points of one call:
// m <= 16 MiB / (4 (ldx + 2 widest hidden layer)) (1,814 points for the
// 257-1024-512-256-128-1 network); larger requests return PIFU_ERR_ARG.
#include <cstring>
#include <mutex>

#include "../../include/pifu.h"
#include "pifu_internal.h"

namespace pifu {
namespace {

constexpr size_t kScratchBytes = 16u << 20;
constexpr int64_t kScratchFloats = (int64_t)(kScratchBytes / sizeof(float));
constexpr int kMaxDevices = 64;
constexpr int kMaxLayers = 16;

static __device__ __align__(256) float g_scratch[kScratchFloats];

// Device address of g_scratch on the current device.  In host code the name
// g_scratch is only a host-side stand-in, never a device address.  Outside a
// stream capture the address is looked up on every call (cheap), so that a
// module reloaded after cudaDeviceReset, or another context made current on
// the same device, is followed; inside a capture the address of the last
// lookup on this device is used (the first call on a device has to come
// before any capture).  The first lookup in a process also loads the
// library's device code and its static arrays onto the device when CUDA loads
// modules lazily (the default since CUDA 12.2): that load allocates the
// 16 MiB array, which is why the first call must come while that much device
// memory is still free.
std::mutex g_mu;
float* g_scratch_dev[kMaxDevices] = {};

int scratch_address(cudaStream_t s, float** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PIFU_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return PIFU_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cs == cudaStreamCaptureStatusNone || !g_scratch_dev[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return PIFU_ERR_CUDA;
        g_scratch_dev[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_dev[dev];
    return PIFU_OK;
}

// Shapes and byte offsets of the occupancy net inside the blob (parsed on
// the host into fixed-size arrays: no heap allocation).
struct BlobNet {
    int d_in = 0, L = 0;
    float slope = 0.f;
    int width[kMaxLayers] = {};
    int fan_in[kMaxLayers] = {};
    int skip[kMaxLayers] = {};
    size_t w_off[kMaxLayers] = {};
    size_t b_off[kMaxLayers] = {};
};

bool rd_u32(const uint8_t* p, size_t n, size_t& off, uint32_t& v) {
    if (off + 4 > n) return false;
    std::memcpy(&v, p + off, 4);
    off += 4;
    return true;
}

int parse_blob_net(const uint8_t* p, size_t n, size_t& off, int want_kind, BlobNet* out) {
    uint32_t kind, d_in, L, slope_bits, skip_mask;
    if (!rd_u32(p, n, off, kind) || !rd_u32(p, n, off, d_in) || !rd_u32(p, n, off, L) ||
        !rd_u32(p, n, off, slope_bits))
        return PIFU_ERR_FORMAT;
    if ((int)kind != want_kind || d_in == 0 || d_in > 4096 || L == 0 || L > (uint32_t)kMaxLayers)
        return PIFU_ERR_FORMAT;
    BlobNet net;
    net.d_in = (int)d_in;
    net.L = (int)L;
    std::memcpy(&net.slope, &slope_bits, 4);
    for (uint32_t l = 0; l < L; ++l) {
        uint32_t w;
        if (!rd_u32(p, n, off, w) || w == 0 || w > 8192) return PIFU_ERR_FORMAT;
        net.width[l] = (int)w;
    }
    if (!rd_u32(p, n, off, skip_mask)) return PIFU_ERR_FORMAT;
    if ((kind == 0 && net.width[L - 1] != 1) || (kind == 1 && net.width[L - 1] != 3))
        return PIFU_ERR_FORMAT;
    for (uint32_t l = 0; l < L; ++l) {
        net.skip[l] = (l > 0) && ((skip_mask >> l) & 1u);
        net.fan_in[l] = (l == 0 ? (int)d_in : net.width[l - 1]) + (net.skip[l] ? (int)d_in : 0);
        net.w_off[l] = off;
        const size_t wb = (size_t)net.width[l] * net.fan_in[l] * 4;
        if (off + wb < off || off + wb > n) return PIFU_ERR_FORMAT;
        off += wb;
        net.b_off[l] = off;
        const size_t bb = (size_t)net.width[l] * 4;
        if (off + bb > n) return PIFU_ERR_FORMAT;
        off += bb;
    }
    if (out) *out = net;
    return PIFU_OK;
}

// Hidden layer straight from the blob's row-major [n_out][fan_in] weights
// (fan_in arbitrary, rows only 4-byte aligned): 64x64 output tiles, 16-deep
// K slices, each thread 4x4 outputs; bias + leaky-ReLU fused.
constexpr int NBM = 64, NBN = 64, NBK = 16;

__global__ void __launch_bounds__(256) blob_layer_kernel(int M, int N, const float* __restrict__ A1,
                                                         int lda1, int K1,
                                                         const float* __restrict__ A2, int lda2,
                                                         int K2, const float* __restrict__ W,
                                                         const float* __restrict__ bias,
                                                         float slope, float* __restrict__ Out,
                                                         int ldo) {
    __shared__ float As[NBK][NBM + 4];
    __shared__ float Ws[NBK][NBN + 4];
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int m0 = blockIdx.y * NBM, n0 = blockIdx.x * NBN;
    const int K = K1 + K2;
    float acc[4][4] = {};
    for (int k0 = 0; k0 < K; k0 += NBK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + 256 * r;
            const int row = e >> 4, kk = e & 15;
            const int k = k0 + kk;
            float a = 0.f;
            if (m0 + row < M && k < K)
                a = (k < K1) ? A1[(int64_t)(m0 + row) * lda1 + k]
                             : A2[(int64_t)(m0 + row) * lda2 + (k - K1)];
            As[kk][row] = a;
            float w = 0.f;
            if (n0 + row < N && k < K) w = W[(int64_t)(n0 + row) * K + k];
            Ws[kk][row] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < NBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Ws[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int row = m0 + ty + 16 * i;
        if (row >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + tx + 16 * j;
            if (col >= N) continue;
            const float o = acc[i][j] + bias[col];
            Out[(int64_t)row * ldo + col] = o >= 0.f ? o : slope * o;
        }
    }
}

}  // namespace
}  // namespace pifu

using namespace pifu;

extern "C" int pifu_query_noalloc(const void* weight_blob, size_t bytes, const void* weight_blob_dev,
                                  const pifu_fmap* occ_map, const float calib[12],
                                  const float* pts_dev, int64_t m, float* occ_dev, void* stream) {
    if (!weight_blob || !weight_blob_dev || !calib || m < 0) return PIFU_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(weight_blob_dev) & 3u) != 0) return PIFU_ERR_ARG;
    // Shapes from the host copy of the blob; both nets are validated.
    const uint8_t* p = static_cast<const uint8_t*>(weight_blob);
    size_t off = 0;
    uint32_t version = 0, n_nets = 0;
    if (bytes < 12 || std::memcmp(p, "PIFU", 4) != 0) return PIFU_ERR_FORMAT;
    off = 4;
    if (!rd_u32(p, bytes, off, version) || version != 1 || !rd_u32(p, bytes, off, n_nets) ||
        n_nets != 2)
        return PIFU_ERR_FORMAT;
    BlobNet net;
    int st = parse_blob_net(p, bytes, off, 0, &net);
    if (st == PIFU_OK) st = parse_blob_net(p, bytes, off, 1, nullptr);
    if (st == PIFU_OK && off != bytes) st = PIFU_ERR_FORMAT;
    if (st != PIFU_OK) return st;
    if (m == 0) return PIFU_OK;
    if (!pts_dev || !occ_dev || !occ_map || !occ_map->data) return PIFU_ERR_ARG;
    if (occ_map->H < 1 || occ_map->W < 1 || occ_map->C < 4 || occ_map->C % 4 != 0 ||
        (reinterpret_cast<uintptr_t>(occ_map->data) & 15u) != 0)
        return PIFU_ERR_ARG;
    if (occ_map->dtype != PIFU_F32) return PIFU_ERR_UNSUPPORTED;
    if (net.d_in != occ_map->C + 1) return PIFU_ERR_ARG;

    // Scratch plan: per point one gather row (ldx floats) and two ping-pong
    // hidden rows.  One call evaluates at most m_max points, the number that
    // fits the fixed 16 MiB array; larger requests are rejected.
    const int ldx = (net.d_in + 7) / 8 * 8;
    int max_hidden = 8;
    for (int l = 0; l + 1 < net.L; ++l) max_hidden = net.width[l] > max_hidden ? net.width[l] : max_hidden;
    const int64_t per_point = ldx + 2 * (int64_t)max_hidden;
    const int64_t m_max = kScratchFloats / per_point;
    if (m > m_max) return PIFU_ERR_ARG;

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* scratch = nullptr;
    st = scratch_address(s, &scratch);
    if (st != PIFU_OK) return st;
    float* X = scratch;
    float* H[2] = {scratch + m * ldx, scratch + m * (ldx + max_hidden)};

    const char* wdev = static_cast<const char*>(weight_blob_dev);
    Calib cal;
    std::memcpy(cal.c, calib, sizeof(cal.c));
    Map map{occ_map->data, occ_map->H, occ_map->W, occ_map->C, occ_map->dtype};
    PointSrc src{PTS_XYZ, pts_dev, nullptr, 0, 0};
    Epilogue epi{};
    epi.mode = EPI_STORE;
    epi.act = ACT_SIGMOID;
    epi.out = occ_dev;
    if (launch_gather(src, 0, m, cal, map, Map{}, X, ldx, s) != cudaSuccess) return PIFU_ERR_CUDA;
    const float* h = nullptr;
    int hw = 0;
    for (int l = 0; l + 1 < net.L; ++l) {
        const int K1 = l == 0 ? 0 : hw;
        const int K2 = (l == 0 || net.skip[l]) ? net.d_in : 0;
        float* out = H[l & 1];
        dim3 grid((net.width[l] + NBN - 1) / NBN, (unsigned)((m + NBM - 1) / NBM));
        blob_layer_kernel<<<grid, 256, 0, s>>>(
            (int)m, net.width[l], h, hw, K1, X, ldx, K2,
            reinterpret_cast<const float*>(wdev + net.w_off[l]),
            reinterpret_cast<const float*>(wdev + net.b_off[l]), net.slope, out, net.width[l]);
        if (cudaGetLastError() != cudaSuccess) return PIFU_ERR_CUDA;
        h = out;
        hw = net.width[l];
    }
    const int l = net.L - 1;
    const int K1 = l == 0 ? 0 : hw;
    const int K2 = (l == 0 || net.skip[l]) ? net.d_in : 0;
    if (launch_last_layer(0, m, 1, h, hw, K1, X, ldx, K2,
                          reinterpret_cast<const float*>(wdev + net.w_off[l]), net.fan_in[l],
                          reinterpret_cast<const float*>(wdev + net.b_off[l]), epi, s) != cudaSuccess)
        return PIFU_ERR_CUDA;
    return PIFU_OK;
}
