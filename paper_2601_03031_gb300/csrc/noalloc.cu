// vc_commit_rows_noalloc: the row commitments C_j of VC.Commit computed without any device
// allocation.  The scratch of the row MSMs (one Jacobian term per input element plus the
// ping-pong half used by the pairwise reduction) lives in a file-scope device array of fixed size.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/flexproofs.h"
#include "k_common.cuh"

namespace {

constexpr uint64_t NOALLOC_MAX_N = 1ull << 14;                    // largest vector accepted
constexpr size_t NOALLOC_SCRATCH_BYTES = (NOALLOC_MAX_N + NOALLOC_MAX_N / 2) * fpk::G1J_BYTES + 256;

// Shared by every call on a device; holds the previous call's contents.  The first 256 bytes are
// the status word (cleared by every call before use), the rest the term and reduction buffers.
static __device__ __align__(256) uint8_t g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_scratch_ptr[MAX_DEVICES] = {};

__global__ void k_noalloc_terms(const fr* m, const g1a* lam, uint64_t n, uint32_t M, g1j* out, uint32_t* err) {
    uint64_t i = fpk::gtid();
    if (i >= n) return;
    fr c = m[i];
    if (!fr_canonical_lt_r(c)) { atomicOr(err, 1u); fr_zero(c); }
    out[i] = g1_mul(lam[i % M], c.v);
}

}  // namespace

namespace fpk {
const void* pp_lambda_top(const fp_pp* pp);     // Lambda_{l_c} (M points), defined with fp_pp
}

extern "C" fp_status vc_commit_rows_noalloc(const fp_pp* pp, const uint64_t* m_dev, uint8_t* rows_dev,
                                            void* stream) {
    if (!pp || !m_dev || !rows_dev) return FP_EINVAL;
    uint32_t log_n = 0, R = 0, M = 0;
    vc_pp_dims(pp, &log_n, &R, &M);
    const uint64_t N = (uint64_t)R * M;
    if (N > NOALLOC_MAX_N) return FP_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return FP_EDEVICE;
    void* base = nullptr;
    {
        // one-time set-up per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FP_EDEVICE;
            g_scratch_ptr[dev] = p;
        }
        base = g_scratch_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t* err = (uint32_t*)base;
    uint8_t* terms = (uint8_t*)base + 256;
    uint8_t* half = terms + NOALLOC_MAX_N * fpk::G1J_BYTES;
    const void* lam = fpk::pp_lambda_top(pp);
    if (cudaMemsetAsync(err, 0, sizeof(uint32_t), s) != cudaSuccess) return FP_EDEVICE;
    FP_KERNEL("k_noalloc_terms", s,
              k_noalloc_terms<<<fpk::grid_for(N, 64), 64, 0, s>>>((const fr*)m_dev, (const g1a*)lam, N, M,
                                                                  (g1j*)terms, err));
    void* a = terms;
    void* b = half;
    for (uint64_t n = N; n > R; n /= 2) {
        fpk::g1_pair_reduce(a, b, n / 2, s);
        void* t = a; a = b; b = t;
    }
    fpk::g1j_to_affine(a, nullptr, rows_dev, fpk::G1_SER, R, s);
    if (cudaGetLastError() != cudaSuccess) return FP_EDEVICE;
    uint32_t herr = 0;
    if (cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FP_EDEVICE;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FP_EDEVICE;
    return herr ? FP_ERANGE : FP_OK;
}
