// C ABI of the FlexProofs GB300 path (declared in include/flexproofs.h): host-side orchestration
// of the kernels on one stream.  No arithmetic of the method runs on the host; the host only
// sizes buffers, enqueues kernels and copies bytes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <chrono>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/flexproofs.h"
#include "kernels.h"

using namespace fpk;

struct fp_pp {
    uint32_t log_n, log_r, log_c, R, M;
    const fp_pp* parent = nullptr;  // views share the parent's tables (all but lam_tab)
    void* lam = nullptr;      // G1 affine, 2M - 1: Lambda_t at offset 2^t - 1
    void* lam_tab = nullptr;  // G1 affine, 2M: Lambda_{l_c} and its GLV partners (MSM bases)
    void* g2w_tab = nullptr;  // G2 affine, 4 x 2R: (-1)^h psi^h(g2^{beta^i}) (W-proof MSM bases)
    void* g2comb = nullptr;   // comb tables of g2^{beta^i}, i < 2R - 1 (W proofs of few blocks; R <= G2_COMB_MAX_R)
    void* lam_comb = nullptr; // comb tables of Lambda_{l_c} (the commit's bases; M <= LAM_COMB_MAX_M), own per view
    void* g1beta = nullptr;   // G1 affine
    void* g2pow = nullptr;    // G2 affine, 2R - 1: g2^{beta^i}
    void* g2tau = nullptr;    // G2 affine, l_c
};

struct fp_commit {
    const fp_pp* pp;
    void* m_canon = nullptr;  // fr canonical, N
    void* m_mont = nullptr;   // fr Montgomery, N
    void* rows = nullptr;     // G1 affine, R
    void* rows_ser = nullptr; // R x 96
    void* C = nullptr;        // fq12
    void* C_ser = nullptr;    // 576
    uint32_t* err = nullptr;  // device word: non-zero if an input value was >= r
    cudaEvent_t done = nullptr;       // C (and everything) ready
    cudaEvent_t rows_done = nullptr;  // m, the row commitments and their serialisation ready
    cudaStream_t stream;
    // completion events of the calls that read this handle on other streams (vc_prove_all); the
    // free waits for them, stream-ordered, without blocking the host
    mutable std::mutex mu;
    mutable std::vector<cudaEvent_t> uses;
};

struct fp_g1_bases {
    uint64_t n;
    void* tab = nullptr;      // G1 affine, 2n: P_i, then -phi(P_i) (the GLV partner)
};

struct fp_proofs {
    const fp_pp* pp;
    ProofLayout L;
    void* rows_ser = nullptr;  // R x 96 (own copy)
    void* blocks = nullptr;    // K x bopen_len
    void* row_tree = nullptr;  // R x (2M - 1) x 32
    void* top_tree = nullptr;  // (2R - 1) x 32
    void* rj = nullptr;        // fr, R
    void* g = nullptr;         // fr Montgomery, (2R - 1) x M
    void* D = nullptr;         // G1 affine, 2R - 1
    void* D_ser = nullptr;     // (2R - 1) x 96
    void* pst_ser = nullptr;   // (M - 1) x 96
    cudaStream_t stream;
    bool step2 = true;         // false: Step 1 only (OpenAll for sub-arrays), no element proofs
    uint32_t k0 = 0, nopen = 0;   // blocks [k0, k0 + nopen) hold their pi_{C_k}
};

namespace {

thread_local std::string g_last_error;

struct CudaError {
    fp_status st;
};

void check(cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
        throw CudaError{e == cudaErrorMemoryAllocation ? FP_ENOMEM : FP_EDEVICE};
    }
}
void check_launch(const char* what) { check(cudaGetLastError(), what); }

void* dalloc(size_t bytes, cudaStream_t s) {
    void* p = nullptr;
    check(cudaMallocAsync(&p, bytes ? bytes : 16, s), "cudaMallocAsync");
    return p;
}
void dfree(void*& p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
}

fp_status device_ok() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        g_last_error = e != cudaSuccess ? cudaGetErrorString(e) : "no CUDA device";
        return FP_EDEVICE;
    }
    return FP_OK;
}

template <typename F>
fp_status guarded(F&& f) {
    fp_status st = device_ok();
    if (st != FP_OK) return st;
    try {
        return f();
    } catch (const CudaError& e) {
        return e.st;
    }
}

// pairwise reduction of `n` consecutive elements down to `target` (n / target a power of two);
// ping-pongs between a and b, returns the buffer holding the result
template <typename Red>
void* reduce_pairs(void* a, void* b, uint64_t n, uint64_t target, Red red, cudaStream_t s) {
    while (n > target) {
        red(a, b, n / 2, s);
        std::swap(a, b);
        n /= 2;
    }
    return a;
}

// the same reduction by block trees (g1_tree_reduce / g2_tree_reduce): a factor of up to gmax per
// launch, for few sums whose pairwise launches would each wait one addition's latency
template <typename Red>
void* reduce_tree(void* a, void* b, uint64_t n, uint64_t target, uint32_t gmax, Red red, cudaStream_t s) {
    while (n > target) {
        const uint32_t gs = (uint32_t)std::min<uint64_t>(gmax, n / target);
        red(a, b, n, gs, s);
        std::swap(a, b);
        n /= gs;
    }
    return a;
}
// sums of few points (one block per sum is enough to fill the GPU's share the round leaves free)
constexpr uint64_t TREE_REDUCE_MAX = 8192;

size_t bopen_len(uint32_t log_r) { return (size_t)log_r * ROUND_BYTES + G1_SER + 2 * G2_SER; }

// Internal non-blocking streams: OpenAll's latency-bound Step 1 runs on three high-priority
// streams (the round chain, and beside it the sparse G1 terms and the shifted fold bases), the
// throughput-bound Step 2 on a low-priority stream; all are forked from and joined back to the caller's stream with events
// created per call.  Each caller stream (per device) gets its own set, so calls on different caller
// streams run concurrently; past 256 caller streams the sets are shared (still correct, less
// concurrent).
struct Streams {
    cudaStream_t hi = nullptr, sp = nullptr, pre = nullptr, la[2] = {nullptr, nullptr}, fold = nullptr, lo = nullptr;
    cudaStream_t tail = nullptr;   // Commit's pairings of the row commitments (high priority)
};
struct StreamKey { int dev; cudaStream_t user; Streams set; };
std::vector<StreamKey> g_sets;
std::mutex g_aux_mu;
Streams make_set() {
    Streams a;
    int lo = 0, hi = 0;
    check(cudaDeviceGetStreamPriorityRange(&lo, &hi), "priority range");
    check(cudaStreamCreateWithPriority(&a.hi, cudaStreamNonBlocking, hi), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.sp, cudaStreamNonBlocking, hi), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.pre, cudaStreamNonBlocking, hi), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.la[0], cudaStreamNonBlocking, hi), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.la[1], cudaStreamNonBlocking, hi), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.fold, cudaStreamNonBlocking, hi), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.lo, cudaStreamNonBlocking, lo), "cudaStreamCreate");
    check(cudaStreamCreateWithPriority(&a.tail, cudaStreamNonBlocking, hi), "cudaStreamCreate");
    return a;
}
Streams streams(cudaStream_t user) {
    int dev = 0;
    check(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_aux_mu);
    size_t same_dev = 0;
    for (auto& e : g_sets) {
        if (e.dev != dev) continue;
        if (e.user == user) return e.set;
        same_dev++;
    }
    if (same_dev >= 256) {                       // share: pick by the stream handle
        size_t pick = (size_t)(((uintptr_t)user >> 4) % same_dev), q = 0;
        for (auto& e : g_sets)
            if (e.dev == dev && q++ == pick) return e.set;
    }
    g_sets.push_back({dev, user, make_set()});
    return g_sets.back().set;
}
cudaEvent_t new_event() {
    cudaEvent_t e = nullptr;
    check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    return e;
}

}  // namespace

namespace {
std::mutex g_limits_mu;
fpk::EngineLimits g_limits;
}  // namespace

namespace fpk {
EngineLimits engine_limits() {
    std::lock_guard<std::mutex> lk(g_limits_mu);
    return g_limits;
}
const void* pp_lambda_top(const fp_pp* pp) { return (const uint8_t*)pp->lam + ((size_t)pp->M - 1) * G1A_BYTES; }
}  // namespace fpk

extern "C" {

const char* fp_strerror(fp_status s) {
    switch (s) {
        case FP_OK: return "ok";
        case FP_EINVAL: return "invalid argument";
        case FP_ENOMEM: return "out of memory";
        case FP_EDEVICE: return "CUDA device error";
        case FP_ETIMEOUT: return "device wait timed out";
        case FP_EVERIFY: return "proof did not verify";
        case FP_ERANGE: return "scalar out of range (>= r)";
    }
    return "unknown status";
}
const char* fp_last_error(void) { return g_last_error.c_str(); }

fp_status vc_setup(uint32_t log_n, uint32_t b, uint64_t seed, void* stream, fp_pp** out) {
    if (!out || log_n < 2 || log_n > 26) return FP_EINVAL;
    return vc_setup_split(log_n / 2, log_n - log_n / 2, b, seed, stream, out);
}

fp_status vc_setup_split(uint32_t log_r, uint32_t log_c, uint32_t b, uint64_t seed, void* stream, fp_pp** out) {
    if (!out || log_r < 1 || log_c < 1 || log_r > 13 || log_r + log_c > 26) return FP_EINVAL;
    const uint32_t log_n = log_r + log_c, R = 1u << log_r, M = 1u << log_c;
    if (b < 1 || b > R) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        fp_pp* pp = new fp_pp{log_n, log_r, log_c, R, M};
        void *trap = nullptr, *lam_s = nullptr, *pow_s = nullptr, *tau_s = nullptr, *beta_s = nullptr;
        try {
            pp->lam = dalloc((2 * (size_t)M - 1) * G1A_BYTES, s);
            pp->g1beta = dalloc(G1A_BYTES, s);
            pp->g2pow = dalloc((2 * (size_t)R - 1) * G2A_BYTES, s);
            pp->g2tau = dalloc((size_t)log_c * G2A_BYTES, s);
            trap = dalloc((log_c + 1) * FR_BYTES, s);
            lam_s = dalloc((2 * (size_t)M - 1) * FR_BYTES, s);
            pow_s = dalloc((2 * (size_t)R - 1) * FR_BYTES, s);
            tau_s = dalloc((size_t)log_c * FR_BYTES, s);
            beta_s = dalloc(FR_BYTES, s);
            setup_trapdoor(seed, (int)log_c, trap, s);
            setup_scalars(trap, (int)log_r, (int)log_c, lam_s, pow_s, tau_s, beta_s, s);
            g1_gen_mul(lam_s, 2 * M - 1, pp->lam, s);
            pp->lam_tab = dalloc(2 * (size_t)M * G1A_BYTES, s);
            check(cudaMemcpyAsync(pp->lam_tab, (uint8_t*)pp->lam + ((size_t)M - 1) * G1A_BYTES, (size_t)M * G1A_BYTES,
                                  cudaMemcpyDeviceToDevice, s), "D2D");
            msm_bases_endo(pp->lam_tab, M, s);
            if (M <= LAM_COMB_MAX_M) {
                pp->lam_comb = dalloc(lam_comb_bytes(M), s);
                void* scr = dalloc(lam_comb_scratch_bytes(M), s);
                lam_comb_tables(pp->lam_tab, M, scr, pp->lam_comb, s);
                dfree(scr, s);
            }
            pp->g2w_tab = dalloc(8 * (size_t)R * G2A_BYTES, s);
            g1_gen_mul(beta_s, 1, pp->g1beta, s);
            g2_gen_mul(pow_s, 2 * R - 1, pp->g2pow, s);
            msm_bases_g2(pp->g2pow, 2 * R - 1, 2 * R, pp->g2w_tab, s);
            if (R <= G2_COMB_MAX_R) {
                pp->g2comb = dalloc(g2_comb_bytes(2 * R - 1), s);
                void* chain = dalloc(g2_comb_chain_bytes(2 * R - 1), s);
                g2_comb_tables(pp->g2pow, 2 * R - 1, chain, pp->g2comb, s);
                dfree(chain, s);
            }
            g2_gen_mul(tau_s, log_c, pp->g2tau, s);
            check_launch("vc_setup kernels");
            // the trapdoor and its scalar tables are cleared before release
            check(cudaMemsetAsync(trap, 0, (log_c + 1) * FR_BYTES, s), "memset");
            check(cudaMemsetAsync(lam_s, 0, (2 * (size_t)M - 1) * FR_BYTES, s), "memset");
            check(cudaMemsetAsync(pow_s, 0, (2 * (size_t)R - 1) * FR_BYTES, s), "memset");
            check(cudaMemsetAsync(tau_s, 0, (size_t)log_c * FR_BYTES, s), "memset");
            check(cudaMemsetAsync(beta_s, 0, FR_BYTES, s), "memset");
            dfree(trap, s); dfree(lam_s, s); dfree(pow_s, s); dfree(tau_s, s); dfree(beta_s, s);
            check(cudaStreamSynchronize(s), "vc_setup");
        } catch (...) {
            cudaStreamSynchronize(s);
            fp_pp_free(pp);
            throw;
        }
        *out = pp;
        return FP_OK;
    });
}

fp_status vc_pp_dims(const fp_pp* pp, uint32_t* log_n, uint32_t* R, uint32_t* M) {
    if (!pp) return FP_EINVAL;
    if (log_n) *log_n = pp->log_n;
    if (R) *R = pp->R;
    if (M) *M = pp->M;
    return FP_OK;
}

fp_status vc_pp_export(const fp_pp* pp, uint8_t* out, size_t cap, size_t* len) {
    if (!pp || !len) return FP_EINVAL;
    size_t n = (2 * (size_t)pp->M - 1) * G1_SER + G1_SER + (2 * (size_t)pp->R - 1) * G2_SER + pp->log_c * G2_SER;
    *len = n;
    if (!out) return FP_OK;
    if (cap < n) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        cudaStream_t s = 0;
        void* d = dalloc(n, s);
        uint8_t* o = (uint8_t*)d;
        g1a_serialize(pp->lam, o, G1_SER, 2 * pp->M - 1, s);
        o += (2 * (size_t)pp->M - 1) * G1_SER;
        g1a_serialize(pp->g1beta, o, G1_SER, 1, s);
        o += G1_SER;
        g2a_serialize(pp->g2pow, o, G2_SER, 2 * pp->R - 1, s);
        o += (2 * (size_t)pp->R - 1) * G2_SER;
        g2a_serialize(pp->g2tau, o, G2_SER, pp->log_c, s);
        check_launch("vc_pp_export");
        check(cudaMemcpyAsync(out, d, n, cudaMemcpyDeviceToHost, s), "D2H");
        dfree(d, s);
        check(cudaStreamSynchronize(s), "vc_pp_export");
        return FP_OK;
    });
}

}  // extern "C"

namespace {
// enqueues VC.Commit on s; the range-check word stays in cm->err and cm->done marks completion
fp_commit* commit_enqueue(const fp_pp* pp, const uint64_t* m, int on_device, cudaStream_t s) {
    const uint32_t R = pp->R, M = pp->M;
    const uint64_t N = (uint64_t)R * M;
    fp_commit* cm = new fp_commit{pp};
    cm->stream = s;
    void *src = nullptr, *t1 = nullptr, *t2 = nullptr, *ml = nullptr, *ml2 = nullptr;
    try {
        cm->m_canon = dalloc(N * FR_BYTES, s);
        cm->m_mont = dalloc(N * FR_BYTES, s);
        cm->rows = dalloc(R * G1A_BYTES, s);
        cm->rows_ser = dalloc(R * G1_SER, s);
        cm->C = dalloc(FQ12_BYTES, s);
        cm->C_ser = dalloc(GT_SER, s);
        cm->err = (uint32_t*)dalloc(sizeof(uint32_t), s);
        check(cudaEventCreateWithFlags(&cm->done, cudaEventDisableTiming), "cudaEventCreate");
        check(cudaEventCreateWithFlags(&cm->rows_done, cudaEventDisableTiming), "cudaEventCreate");
        check(cudaMemsetAsync(cm->err, 0, sizeof(uint32_t), s), "memset");
        const void* msrc = m;
        if (!on_device) {
            src = dalloc(N * FR_BYTES, s);
            check(cudaMemcpyAsync(src, m, N * FR_BYTES, cudaMemcpyHostToDevice, s), "H2D m");
            msrc = src;
        }
        load_vector(msrc, N, cm->m_canon, cm->m_mont, cm->err, s);
        // C_j = sum_a m[jM + a] Lambda_{l_c}[a]: R sums of M terms over the shared bases, from their
        // comb tables when the setup has them (partial sums per base and quarter of the windows,
        // reduced pairwise and then by block trees), else R MSMs
        if (pp->lam_comb) {
            const uint64_t np = (uint64_t)R * M * lam_comb_parts();
            t1 = dalloc(np * G1J_BYTES, s);
            t2 = dalloc((np / 2 + 1) * G1J_BYTES, s);
            lam_comb_partials(pp->lam_comb, cm->m_canon, R, M, t1, s);
            void* r1 = reduce_pairs(t1, t2, np, std::min<uint64_t>(np, (uint64_t)R * 32), g1_pair_reduce, s);
            void* r2 = reduce_tree(r1, r1 == t1 ? t2 : t1, std::min<uint64_t>(np, (uint64_t)R * 32), R, 32,
                                   g1_tree_reduce, s);
            g1j_to_affine(r2, cm->rows, cm->rows_ser, G1_SER, R, s);
        } else {
            const MsmShape sh = msm_shape(M, R, M, fp_msm_window(M, R));
            t1 = dalloc(msm_scratch_bytes(sh), s);
            msm_g1(pp->lam_tab, cm->m_canon, sh, t1, cm->rows, cm->rows_ser, s);
        }
        // C = prod_j e(C_j, v_j): R Miller loops, pairwise products, one final exponentiation, on an
        // internal stream after the rows: the caller's stream goes on (OpenAll's pairings and Step 2
        // need the rows only), cm->done marks C
        ml = dalloc(R * FQ12_BYTES, s);
        ml2 = dalloc((R / 2 + 1) * FQ12_BYTES, s);
        check(cudaEventRecord(cm->rows_done, s), "event");
        cudaStream_t st = streams(s).tail;
        check(cudaStreamWaitEvent(st, cm->rows_done, 0), "wait");
        commit_miller(cm->rows, pp->g2pow, R, ml, st);
        void* prod = reduce_pairs(ml, ml2, R, 1, fq12_pair_reduce, st);
        final_exp_group(prod, 1, cm->C, cm->C_ser, 1, GT_SER, 0, st);
        check_launch("vc_commit kernels");
        dfree(src, s); dfree(t1, s); dfree(t2, s); dfree(ml, st); dfree(ml2, st);
        check(cudaEventRecord(cm->done, st), "event");
    } catch (...) {
        cudaDeviceSynchronize();                     // the caller's stream and the internal one
        dfree(src, s); dfree(t1, s); dfree(t2, s); dfree(ml, s); dfree(ml2, s);
        fp_commit_free(cm);
        throw;
    }
    return cm;
}

fp_status commit_status(const fp_commit* cm) {
    uint32_t herr = 0;
    check(cudaEventSynchronize(cm->done), "vc_commit");
    check(cudaMemcpy(&herr, cm->err, sizeof herr, cudaMemcpyDeviceToHost), "D2H err");
    return herr ? FP_ERANGE : FP_OK;
}
}  // namespace

extern "C" {

fp_status vc_commit(const fp_pp* pp, const uint64_t* m, int on_device, void* stream, fp_commit** out) {
    if (!pp || !m || !out) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        fp_commit* cm = commit_enqueue(pp, m, on_device, (cudaStream_t)stream);
        fp_status st;
        try {
            st = commit_status(cm);
        } catch (...) {
            fp_commit_free(cm);
            throw;
        }
        if (st != FP_OK) {
            fp_commit_free(cm);
            return st;
        }
        *out = cm;
        return FP_OK;
    });
}

fp_status vc_commit_async(const fp_pp* pp, const uint64_t* m, int on_device, void* stream, fp_commit** out) {
    if (!pp || !m || !out) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        *out = commit_enqueue(pp, m, on_device, (cudaStream_t)stream);
        return FP_OK;
    });
}

fp_status vc_commit_status(const fp_commit* cm) {
    if (!cm) return FP_EINVAL;
    return guarded([&]() -> fp_status { return commit_status(cm); });
}

fp_status vc_pp_view(const fp_pp* pp, uint32_t log_n, fp_pp** out) {
    if (!pp || !out || log_n < 2 || log_n > pp->log_n) return FP_EINVAL;
    return vc_pp_view_split(pp, log_n / 2, log_n - log_n / 2, out);
}

fp_status vc_pp_view_split(const fp_pp* pp, uint32_t log_r, uint32_t log_c, fp_pp** out) {
    if (!pp || !out || log_r < 1 || log_c < 1) return FP_EINVAL;
    const fp_pp* root = pp->parent ? pp->parent : pp;
    if (log_r > root->log_r || log_c > root->log_c) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        const uint32_t log_n = log_r + log_c, R = 1u << log_r, M = 1u << log_c;
        fp_pp* v = new fp_pp{log_n, log_r, log_c, R, M};
        v->parent = root;
        v->lam = root->lam;                 // Lambda_t for t <= l_c are the same prefix levels
        v->g1beta = root->g1beta;
        v->g2pow = root->g2pow;             // g2^{beta^i}, i < 2R - 1: a prefix
        v->g2tau = root->g2tau;             // tau_0 .. tau_{l_c - 1}: a prefix
        v->g2comb = root->g2comb;           // the tables of a prefix of g2pow
        cudaStream_t s = 0;
        try {
            v->lam_tab = dalloc(2 * (size_t)M * G1A_BYTES, s);
            check(cudaMemcpyAsync(v->lam_tab, (uint8_t*)root->lam + ((size_t)M - 1) * G1A_BYTES, (size_t)M * G1A_BYTES,
                                  cudaMemcpyDeviceToDevice, s), "D2D");
            msm_bases_endo(v->lam_tab, M, s);
            if (M <= LAM_COMB_MAX_M) {
                v->lam_comb = dalloc(lam_comb_bytes(M), s);
                void* scr = dalloc(lam_comb_scratch_bytes(M), s);
                lam_comb_tables(v->lam_tab, M, scr, v->lam_comb, s);
                dfree(scr, s);
            }
            v->g2w_tab = dalloc(8 * (size_t)R * G2A_BYTES, s);
            msm_bases_g2(v->g2pow, 2 * R - 1, 2 * R, v->g2w_tab, s);
            check_launch("vc_pp_view");
            check(cudaStreamSynchronize(s), "vc_pp_view");
        } catch (...) {
            cudaStreamSynchronize(s);
            fp_pp_free(v);
            throw;
        }
        *out = v;
        return FP_OK;
    });
}

fp_status vc_commit_get(const fp_commit* cm, uint8_t* gt576, uint8_t* rows) {
    if (!cm) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        cudaStream_t s = cm->stream;
        if (cm->done) check(cudaStreamWaitEvent(s, cm->done, 0), "wait");
        if (gt576) check(cudaMemcpyAsync(gt576, cm->C_ser, GT_SER, cudaMemcpyDeviceToHost, s), "D2H");
        if (rows) check(cudaMemcpyAsync(rows, cm->rows_ser, cm->pp->R * G1_SER, cudaMemcpyDeviceToHost, s), "D2H");
        check(cudaStreamSynchronize(s), "vc_commit_get");
        return FP_OK;
    });
}

}  // extern "C"

namespace {
// Step 1's device buffers for Kc blocks of R rows: FC.BOpen state (A, v, b per block), the round
// outputs, the challenges and the fast-verification proof of v_l
struct Step1Bufs {
    void *A, *v, *bvec, *xprev, *x_mont, *xinv_mont, *xinv_all, *ml, *ml2, *sp, *sp2, *pcoef, *q;
    void* comb = nullptr;                // comb tables of rounds with few points (step1_fold_pre)
    uint32_t comb_n = 0;                 // points they hold
    void *wt = nullptr, *wt2 = nullptr, *wscr = nullptr;
    MsmShape wsh{};
    bool w_msm = false;
};
template <class Alloc>
Step1Bufs step1_bufs(const fp_pp* pp, uint32_t Kc, Alloc&& T) {
    const uint32_t R = pp->R;
    const uint64_t KR = (uint64_t)Kc * R;
    Step1Bufs B;
    B.A = T(KR * G1A_BYTES);
    B.v = T(KR * G2A_BYTES);
    B.bvec = T(KR * FR_BYTES);
    B.xprev = T(Kc * 32);
    B.x_mont = T(2 * Kc * FR_BYTES);        // two rounds' challenges (the look-ahead schedule alternates)
    B.xinv_mont = T(2 * Kc * FR_BYTES);
    B.xinv_all = T((size_t)Kc * pp->log_r * FR_BYTES);
    B.ml = T(KR * FQ12_BYTES);
    B.ml2 = T((KR / 2 + 1) * FQ12_BYTES);
    B.sp = T(KR * G1J_BYTES);
    B.sp2 = T((KR / 2 + 1) * G1J_BYTES);
    B.pcoef = T((size_t)Kc * (2 * R - 1) * FR_BYTES);
    B.q = T((size_t)Kc * 2 * R * FR_BYTES);
    B.comb_n = (uint32_t)std::min<uint64_t>(FOLD_COMB_MAX, KR / 2);
    if (B.comb_n) B.comb = T(fold_comb_bytes(B.comb_n));
    // W proofs: one batched G2 MSM over the shared bases g2^{beta^i} when many blocks share them,
    // else one scalar multiplication per term and pairwise sums (with few batches the MSM's bucket
    // reduction runs nearly serially per window)
    B.w_msm = KR * 2 > 4096 && Kc >= 8;
    if (B.w_msm) {
        B.wsh = msm_shape(2 * R, Kc, 2 * R, fp_msm_window_g2(2 * R, Kc), 4, 65);
        B.wscr = T(msm_scratch_bytes_g2(B.wsh));
    } else {
        B.wt = T((size_t)Kc * 2 * R * G2J_BYTES);
        B.wt2 = T(((size_t)Kc * R + 1) * G2J_BYTES);
    }
    return B;
}

// Look-ahead buffers (lookahead.cuh) for Kc blocks of R rows, one set per parity of the round (two
// rounds' look-aheads run at once, on two streams): a snapshot of round j-1's state, the Miller
// values by class and their pairwise products (8 Kc h2 <= 2 Kc R), the final exponentiations, affine
// G1 sums and shifted bases, the G1 terms (6 Kc 4 h2 <= 6 Kc R) and their pairwise sums; and the
// exponentiation parts, used on the challenge stream only
struct LaBufs {
    void *A[2], *v[2], *bvec[2], *ml[2], *ml2[2], *fe[2], *gpre[2], *acc[2], *acc2[2], *sp[2], *sp2[2], *pwp;
};
template <class Alloc>
LaBufs la_bufs(const fp_pp* pp, uint32_t Kc, Alloc&& T) {
    const uint64_t KR = (uint64_t)Kc * pp->R;
    LaBufs L;
    for (int i = 0; i < 2; i++) {
        L.A[i] = T(KR * G1A_BYTES);
        L.v[i] = T(KR * G2A_BYTES);
        L.bvec[i] = T(KR * FR_BYTES);
        L.ml[i] = T(2 * KR * FQ12_BYTES);
        L.ml2[i] = T((KR + 1) * FQ12_BYTES);
        L.fe[i] = T((size_t)8 * Kc * FQ12_BYTES);
        L.gpre[i] = T((size_t)12 * Kc * FQ12_BYTES);
        L.acc[i] = T((size_t)6 * Kc * G1A_BYTES);
        L.acc2[i] = T((size_t)12 * Kc * G1A_BYTES);
        L.sp[i] = T(6 * KR * G1J_BYTES);
        L.sp2[i] = T((3 * KR + 1) * G1J_BYTES);
    }
    L.pwp = T((size_t)16 * Kc * FQ12_BYTES);
    return L;
}

// FC.BOpen rounds (Sec. 3, Eq. folding) and the fast-verification proof of v_l for the Kc blocks
// k0 .. k0 + Kc - 1 of size b, whose combined vectors are in B.bvec (their support is the block):
// the round chain on s1, each round's G1 parts on s3 (joined before the challenge) and, in rounds
// with few points, the shifted fold bases on s4 (joined before the fold); the records go to
// blocks1 (stride blen).  s3 must already be ordered after whatever filled B.bvec.
void step1_rounds(const fp_pp* pp, uint32_t k0, uint32_t Kc, uint32_t b, const Step1Bufs& B, uint8_t* blocks1,
                  size_t blen, cudaStream_t s1, cudaStream_t s3, cudaStream_t s4) {
    const uint32_t R = pp->R;
    const int lr = (int)pp->log_r;
    cudaEvent_t ev_folded = new_event(), ev_sparse = new_event(), ev_pre = new_event();
    for (int j = 1; j <= lr; j++) {
        const uint32_t h = R >> j;
        check(cudaEventRecord(ev_folded, s1), "event");
        const bool split = (uint64_t)Kc * h <= B.comb_n;
        if (split) {
            check(cudaStreamWaitEvent(s4, ev_folded, 0), "wait");
            step1_fold_pre(B.A, B.v, B.comb, B.comb_n, Kc, R, h, s4);
            check(cudaEventRecord(ev_pre, s4), "event");
        }
        check(cudaStreamWaitEvent(s3, ev_folded, 0), "wait");
        step1_sparse_terms(B.A, B.bvec, k0, Kc, R, h, b, B.sp, s3);
        void* spr = (uint64_t)Kc * 2 * h <= TREE_REDUCE_MAX
                        ? reduce_tree(B.sp, B.sp2, (uint64_t)Kc * 2 * h, (uint64_t)Kc * 2, 32, g1_tree_reduce, s3)
                        : reduce_pairs(B.sp, B.sp2, (uint64_t)Kc * 2 * h, (uint64_t)Kc * 2, g1_pair_reduce, s3);
        step1_g1_out(spr, Kc, j, blocks1, blen, s3);
        check(cudaEventRecord(ev_sparse, s3), "event");
        const uint64_t nml = step1_miller_g(B.A, B.v, Kc, R, h, B.ml, s1);
        void* mlr = reduce_pairs(B.ml, B.ml2, nml, (uint64_t)Kc * 2, fq12_pair_reduce, s1);
        step1_gt_out(mlr, Kc, j, blocks1, blen, s1);
        check(cudaStreamWaitEvent(s1, ev_sparse, 0), "wait");
        step1_challenge(blocks1, blen, Kc, j, B.xprev, B.x_mont, B.xinv_mont, B.xinv_all, lr, s1);
        if (split) check(cudaStreamWaitEvent(s1, ev_pre, 0), "wait");
        step1_fold(B.A, B.v, B.bvec, B.x_mont, B.xinv_mont, Kc, R, h, split ? B.comb : nullptr, B.comb_n, s1);
    }
    step1_kzg(B.A, B.v, B.xprev, B.xinv_all, Kc, R, lr, blocks1, blen, B.pcoef, B.q, s1);
    uint8_t* w_out = blocks1 + (size_t)lr * ROUND_BYTES + G1_SER + G2_SER;
    if (B.w_msm) {
        msm_g2(pp->g2w_tab, B.q, B.wsh, B.wscr, nullptr, w_out, blen, s1);
    } else {
        if (pp->g2comb) step1_w_comb(pp->g2comb, B.q, Kc, R, B.wt, s1);
        else step1_w_terms(pp->g2pow, B.q, Kc, R, B.wt, s1);
        void* wr = (uint64_t)Kc * 2 * R <= TREE_REDUCE_MAX
                       ? reduce_tree(B.wt, B.wt2, (uint64_t)Kc * 2 * R, Kc, 16, g2_tree_reduce, s1)
                       : reduce_pairs(B.wt, B.wt2, (uint64_t)Kc * 2 * R, Kc, g2_pair_reduce, s1);
        g2j_to_affine(wr, nullptr, w_out, blen, Kc, s1);
    }
    cudaEventDestroy(ev_folded);
    cudaEventDestroy(ev_sparse);
    cudaEventDestroy(ev_pre);
}

// The rounds with look-ahead (lookahead.cuh): round 1 as in step1_rounds; for j >= 2 round j's record
// comes from round j-1's state S_{j-1} and x_{j-1}.  Round j's look-ahead (a snapshot of S_{j-1}, then
// its Miller loops, final exponentiations, G1 sums and shifted bases) starts as soon as round j-2's
// fold has produced S_{j-1}, on look-ahead stream j mod 2 with the buffers of that parity, so the
// look-aheads of consecutive rounds overlap; once x_{j-1} is known only the GT exponentiations by
// x_{j-1}^(+-1), the G1 multiplications and the challenge remain, on the challenge stream s1.  Round
// j-1's fold runs on sF after x_{j-1} and round j's snapshot.  Challenges alternate between two
// buffers (B.x_mont, B.xinv_mont hold 2 Kc entries); a fold still reading x_{j-1} never meets x_{j+1},
// because x_{j+1} waits for round j+1's look-ahead, which waits for that fold.  Streams: s1 challenges,
// s3 round 1's sparse G1 terms, s4 the shifted fold bases, sL[0..1] the look-aheads, sF the folds;
// s3 must already be ordered after whatever filled B.bvec, s1 after B.A and B.v.
void step1_rounds_la(const fp_pp* pp, uint32_t k0, uint32_t Kc, uint32_t b, const Step1Bufs& B,
                     const LaBufs& L, uint8_t* blocks1, size_t blen, cudaStream_t s1, cudaStream_t s3,
                     cudaStream_t s4, const cudaStream_t* sL, cudaStream_t sF) {
    const uint32_t R = pp->R;
    const int lr = (int)pp->log_r;
    const uint64_t KR = (uint64_t)Kc * R;
    auto xm = [&](int j) { return (uint8_t*)B.x_mont + (size_t)(j & 1) * Kc * FR_BYTES; };
    auto xim = [&](int j) { return (uint8_t*)B.xinv_mont + (size_t)(j & 1) * Kc * FR_BYTES; };
    std::vector<cudaEvent_t> evs;
    auto ev = [&]() { evs.push_back(new_event()); return evs.back(); };
    auto wait = [&](cudaStream_t st, cudaEvent_t e) { check(cudaStreamWaitEvent(st, e, 0), "wait"); };
    auto rec = [&](cudaStream_t st) { cudaEvent_t e = ev(); check(cudaEventRecord(e, st), "event"); return e; };
    std::vector<cudaEvent_t> ev_S(lr + 2, nullptr), ev_snap(lr + 2, nullptr), ev_la(lr + 2, nullptr),
        ev_pre(lr + 2, nullptr), ev_x(lr + 2, nullptr);

    // round j's look-ahead from the state S_{j-1} (the caller has ordered sL[j & 1] after it)
    auto lookahead = [&](int j) {
        const int q = j & 1;
        const cudaStream_t st = sL[q];
        const uint32_t h2 = R >> j;
        check(cudaMemcpyAsync(L.A[q], B.A, KR * G1A_BYTES, cudaMemcpyDeviceToDevice, st), "D2D");
        check(cudaMemcpyAsync(L.v[q], B.v, KR * G2A_BYTES, cudaMemcpyDeviceToDevice, st), "D2D");
        check(cudaMemcpyAsync(L.bvec[q], B.bvec, KR * FR_BYTES, cudaMemcpyDeviceToDevice, st), "D2D");
        ev_snap[j] = rec(st);
        la_miller(L.A[q], L.v[q], Kc, R, h2, L.ml[q], st);
        void* mlr = reduce_pairs(L.ml[q], L.ml2[q], (uint64_t)Kc * 8 * h2, (uint64_t)Kc * 8, fq12_pair_reduce, st);
        final_exp_group(mlr, 8 * Kc, L.fe[q], nullptr, 1, 0, 0, st);
        check(cudaMemsetAsync(L.sp[q], 0, (size_t)Kc * 6 * 4 * h2 * G1J_BYTES, st), "memset");
        la_sparse(L.A[q], L.bvec[q], k0, Kc, R, h2, b, L.sp[q], st);
        void* spr = reduce_pairs(L.sp[q], L.sp2[q], (uint64_t)Kc * 24 * h2, (uint64_t)Kc * 6, g1_pair_reduce, st);
        g1j_to_affine(spr, L.acc[q], nullptr, 0, (uint64_t)Kc * 6, st);
        la_pre(L.fe[q], L.acc[q], Kc, L.gpre[q], L.acc2[q], st);
        ev_la[j] = rec(st);
    };
    // round j's fold on sF (after x_j, the shifted bases and the snapshot of S_j for round j + 1)
    auto fold = [&](int j) {
        const uint32_t h = R >> j;
        const bool split = (uint64_t)Kc * h <= B.comb_n;
        wait(sF, ev_x[j]);
        if (split) wait(sF, ev_pre[j]);
        if (j + 1 <= lr) wait(sF, ev_snap[j + 1]);
        step1_fold(B.A, B.v, B.bvec, xm(j), xim(j), Kc, R, h, split ? B.comb : nullptr, B.comb_n, sF);
        ev_S[j + 1] = rec(sF);
    };
    auto fold_pre = [&](int j, cudaEvent_t ready) {
        const uint32_t h = R >> j;
        if ((uint64_t)Kc * h > B.comb_n) return;
        wait(s4, ready);
        step1_fold_pre(B.A, B.v, B.comb, B.comb_n, Kc, R, h, s4);
        ev_pre[j] = rec(s4);
    };

    cudaEvent_t ev_a = rec(s1), ev_b = rec(s3);     // S_1: A, v (s1) and b (s3)
    if (lr >= 2) {
        wait(sL[0], ev_a);
        wait(sL[0], ev_b);
        lookahead(2);
    }
    fold_pre(1, ev_a);
    {   // round 1, direct
        const uint32_t h = R >> 1;
        step1_sparse_terms(B.A, B.bvec, k0, Kc, R, h, b, B.sp, s3);
        void* spr = (uint64_t)Kc * 2 * h <= TREE_REDUCE_MAX
                        ? reduce_tree(B.sp, B.sp2, (uint64_t)Kc * 2 * h, (uint64_t)Kc * 2, 32, g1_tree_reduce, s3)
                        : reduce_pairs(B.sp, B.sp2, (uint64_t)Kc * 2 * h, (uint64_t)Kc * 2, g1_pair_reduce, s3);
        step1_g1_out(spr, Kc, 1, blocks1, blen, s3);
        cudaEvent_t ev_sp = rec(s3);
        const uint64_t nml = step1_miller_g(B.A, B.v, Kc, R, h, B.ml, s1);
        void* mlr = reduce_pairs(B.ml, B.ml2, nml, (uint64_t)Kc * 2, fq12_pair_reduce, s1);
        step1_gt_out(mlr, Kc, 1, blocks1, blen, s1);
        wait(s1, ev_sp);
        step1_challenge(blocks1, blen, Kc, 1, B.xprev, xm(1), xim(1), B.xinv_all, lr, s1);
        ev_x[1] = rec(s1);
    }
    fold(1);
    for (int j = 2; j <= lr; j++) {
        if (j + 1 <= lr) {
            wait(sL[(j + 1) & 1], ev_S[j]);
            lookahead(j + 1);
        }
        fold_pre(j, ev_S[j]);
        wait(s1, ev_la[j]);
        la_gt(L.fe[j & 1], L.gpre[j & 1], xm(j - 1), xim(j - 1), Kc, L.pwp, s1);
        la_out(L.fe[j & 1], L.pwp, L.acc[j & 1], L.acc2[j & 1], xm(j - 1), xim(j - 1), Kc, j, blocks1, blen, s1);
        step1_challenge(blocks1, blen, Kc, j, B.xprev, xm(j), xim(j), B.xinv_all, lr, s1);
        ev_x[j] = rec(s1);
        fold(j);
    }
    wait(s1, ev_S[lr + 1]);
    step1_kzg(B.A, B.v, B.xprev, B.xinv_all, Kc, R, lr, blocks1, blen, B.pcoef, B.q, s1);
    uint8_t* w_out = blocks1 + (size_t)lr * ROUND_BYTES + G1_SER + G2_SER;
    if (B.w_msm) {
        msm_g2(pp->g2w_tab, B.q, B.wsh, B.wscr, nullptr, w_out, blen, s1);
    } else {
        if (pp->g2comb) step1_w_comb(pp->g2comb, B.q, Kc, R, B.wt, s1);
        else step1_w_terms(pp->g2pow, B.q, Kc, R, B.wt, s1);
        void* wr = (uint64_t)Kc * 2 * R <= TREE_REDUCE_MAX
                       ? reduce_tree(B.wt, B.wt2, (uint64_t)Kc * 2 * R, Kc, 16, g2_tree_reduce, s1)
                       : reduce_pairs(B.wt, B.wt2, (uint64_t)Kc * 2 * R, Kc, g2_pair_reduce, s1);
        g2j_to_affine(wr, nullptr, w_out, blen, Kc, s1);
    }
    for (cudaEvent_t e : evs) cudaEventDestroy(e);
}

// Step-1 schedule of the library (fp_set_schedule); the records are the same either way
std::atomic<int> g_schedule{FP_SCHEDULE_DIRECT};
bool lookahead_on(int log_r) { return g_schedule.load(std::memory_order_relaxed) == FP_SCHEDULE_LOOKAHEAD && log_r >= 2; }

// OpenAll's work with Step 1 restricted to the blocks [k0, k0 + Kc) (all blocks: k0 = 0, Kc = K):
// their records are written at their places in the K-block array; Step 2 runs in full.
fp_proofs* prove_impl(const fp_pp* pp, const fp_commit* cm, uint32_t b, uint32_t k0, uint32_t Kc, cudaStream_t s,
                      bool track_use = true, bool with_step2 = true) {
    const uint32_t R = pp->R, M = pp->M;
    {
        const int lr = (int)pp->log_r, lc = (int)pp->log_c;
        const uint32_t K = (R + b - 1) / b;
        fp_proofs* pf = new fp_proofs{pp};
        pf->stream = s;
        pf->L = ProofLayout{R, M, b, K, (int)pp->log_n, lr, lc, bopen_len(pp->log_r)};
        pf->step2 = with_step2;
        pf->k0 = k0;
        pf->nopen = Kc;
        const size_t blen = pf->L.bopen_len;
        uint8_t* blocks1 = nullptr;
        std::vector<void*> tmp;
        auto T = [&](size_t bytes) { void* p = dalloc(bytes, s); tmp.push_back(p); return p; };
        try {
            // the commitment may have been made on another stream: order after its rows (C, which only
            // the statement hashes read, is awaited on their stream)
            if (track_use && (cm->rows_done || cm->done))
                check(cudaStreamWaitEvent(s, cm->rows_done ? cm->rows_done : cm->done, 0), "wait");
            pf->rows_ser = dalloc(R * G1_SER, s);
            check(cudaMemcpyAsync(pf->rows_ser, cm->rows_ser, R * G1_SER, cudaMemcpyDeviceToDevice, s), "D2D");
            pf->blocks = dalloc(K * blen, s);
            blocks1 = (uint8_t*)pf->blocks + (size_t)k0 * blen;
            // Step 2 depends only on the commitment: it runs on a second stream, concurrently with Step 1
            const uint64_t half = M / 2;
            void *pt = nullptr, *pt2 = nullptr;
            if (with_step2) {
                pf->row_tree = dalloc((size_t)R * (2 * M - 1) * DIGEST, s);
                pf->top_tree = dalloc((2 * (size_t)R - 1) * DIGEST, s);
                pf->rj = dalloc(R * FR_BYTES, s);
                pf->g = dalloc((2 * (size_t)R - 1) * M * FR_BYTES, s);
                pf->D = dalloc((2 * (size_t)R - 1) * G1A_BYTES, s);
                pf->D_ser = dalloc((2 * (size_t)R - 1) * G1_SER, s);
                pf->pst_ser = dalloc(((size_t)M - 1) * G1_SER, s);
                pt = T((size_t)lc * half * G1J_BYTES);
                pt2 = T((half / 2 + 1) * G1J_BYTES);
            }
            // every buffer is allocated (stream-ordered on s) before the fork to the internal streams
            const Step1Bufs B = step1_bufs(pp, Kc, T);
            const bool la = lookahead_on(lr);
            const LaBufs L = la ? la_bufs(pp, Kc, T) : LaBufs{};
            void* hstmt = T(Kc * DIGEST);
            void* hscr = T(stmt_hash_scratch_bytes(Kc, R, b));
            const Streams st = streams(s);
            cudaStream_t s2 = st.lo, s1 = st.hi, s3 = st.sp;
            cudaEvent_t ev_fork = new_event(), ev_join = new_event(), ev_join1 = new_event();
            check(cudaEventRecord(ev_fork, s), "event");
            check(cudaStreamWaitEvent(s2, ev_fork, 0), "wait");
            check(cudaStreamWaitEvent(s1, ev_fork, 0), "wait");
            // ---------------- Step 2: Merkle tree, randomise, fold tree, HyperEval (stream s2)
            if (with_step2) {
                step2_leaves(cm->m_canon, R, M, pf->row_tree, s2);
                for (int l = 1; l <= lc; l++) tree_level(pf->row_tree, R, M, l, s2);
                step2_row_leaves(pf->row_tree, cm->rows_ser, R, M, pf->top_tree, s2);
                for (int l = 1; l <= lr; l++) tree_level(pf->top_tree, 1, R, l, s2);
                step2_rj(pf->top_tree, R, pf->rj, s2);
                step2_randomize(cm->m_mont, pf->rj, R, M, pf->g, s2);
                step2_d0(cm->rows, pf->rj, R, pf->D, s2);
                for (int h = 1; h <= lr; h++) {
                    step2_fold_g(pf->g, R, M, h, s2);
                    step2_fold_d(pf->D, R, h, s2);
                }
                g1a_serialize(pf->D, pf->D_ser, G1_SER, 2 * (uint64_t)R - 1, s2);
                step2_pst_terms(pf->g, pp->lam, R, M, lc, pt, s2);
                size_t pst_off = 0;
                for (int t = 0; t < lc; t++) {
                    void* lvl = (uint8_t*)pt + (size_t)t * half * G1J_BYTES;
                    uint64_t nseg = half >> t;
                    void* res = reduce_pairs(lvl, pt2, half, nseg, g1_pair_reduce, s2);
                    g1j_to_affine(res, nullptr, (uint8_t*)pf->pst_ser + pst_off * G1_SER, G1_SER, nseg, s2);
                    pst_off += nseg;
                }
            }
            check(cudaEventRecord(ev_join, s2), "event");

            // ---------------- Step 1: FC.BOpen on every block (Protocol 1, Step 1)
            // round chain on s1; each round's sparse G1 terms on s3, overlapping its Miller loops and
            // final exponentiations, joined before the challenge
            cudaEvent_t ev_init = new_event();
            step1_init(cm->rows, pp->g2pow, Kc, R, B.A, B.v, B.bvec, s1);
            // the statement hashes and r_a only feed b: they run on s3 ahead of the first sparse terms
            // while s1 starts the first round's Miller loops
            check(cudaEventRecord(ev_init, s1), "event");
            check(cudaStreamWaitEvent(s3, ev_init, 0), "wait");
            if (track_use && cm->done) check(cudaStreamWaitEvent(s3, cm->done, 0), "wait");
            step1_stmt_hash(cm->C_ser, cm->rows_ser, k0, Kc, R, b, hscr, hstmt, s3);
            step1_block_r(hstmt, k0, Kc, R, b, B.bvec, s3);
            if (la) step1_rounds_la(pp, k0, Kc, b, B, L, blocks1, blen, s1, s3, st.pre, st.la, st.fold);
            else step1_rounds(pp, k0, Kc, b, B, blocks1, blen, s1, s3, st.pre);
            check(cudaEventRecord(ev_join1, s1), "event");
            check(cudaStreamWaitEvent(s, ev_join1, 0), "join");
            cudaEventDestroy(ev_init);
            cudaEventDestroy(ev_join1);
            check_launch("step 1 kernels");
            check(cudaStreamWaitEvent(s, ev_join, 0), "join");
            cudaEventDestroy(ev_fork);
            cudaEventDestroy(ev_join);
            if (track_use) {
                cudaEvent_t used = new_event();
                check(cudaEventRecord(used, s), "event");
                std::lock_guard<std::mutex> lk(cm->mu);
                cm->uses.push_back(used);
            }
            check_launch("step 2 kernels");
            for (void* p : tmp) cudaFreeAsync(p, s);
            tmp.clear();
        } catch (...) {
            for (void* p : tmp) cudaFreeAsync(p, s);
            cudaStreamSynchronize(s);
            fp_proofs_free(pf);
            throw;
        }
        return pf;
    }
}
}  // namespace

extern "C" {

static_assert(sizeof(fp_engine_limits) == sizeof(fpk::EngineLimits), "engine limits layout");
fp_status fp_engine_limits_default(fp_engine_limits* out) {
    if (!out) return FP_EINVAL;
    const fpk::EngineLimits d;
    std::memcpy(out, &d, sizeof d);
    return FP_OK;
}
fp_status fp_set_engine_limits(const fp_engine_limits* lim) {
    fpk::EngineLimits v;
    if (lim) {
        std::memcpy(&v, lim, sizeof v);
        if (!v.msm_chunks || !v.msm_segment_threads) return FP_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_limits_mu);
    g_limits = v;
    return FP_OK;
}
fp_status fp_get_engine_limits(fp_engine_limits* out) {
    if (!out) return FP_EINVAL;
    const fpk::EngineLimits v = fpk::engine_limits();
    std::memcpy(out, &v, sizeof v);
    return FP_OK;
}

fp_status fp_set_schedule(int schedule) {
    if (schedule != FP_SCHEDULE_DIRECT && schedule != FP_SCHEDULE_LOOKAHEAD) return FP_EINVAL;
    g_schedule.store(schedule, std::memory_order_relaxed);
    return FP_OK;
}
int fp_get_schedule(void) { return g_schedule.load(std::memory_order_relaxed); }

fp_status vc_prove_all(const fp_pp* pp, const fp_commit* cm, uint32_t b, void* stream, fp_proofs** out) {
    if (!pp || !cm || !out || cm->pp != pp) return FP_EINVAL;
    if (b < 1 || b > pp->R) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        *out = prove_impl(pp, cm, b, 0, (pp->R + b - 1) / b, (cudaStream_t)stream);
        return FP_OK;
    });
}

}  // extern "C"

namespace {
// host wall-clock phases of this thread's last vc_prove_all_batch call (fp_batch_last_times)
struct BatchTimes { double capture_ms = 0, instantiate_ms = 0, run_ms = 0; };
thread_local BatchTimes g_batch_times;
}  // namespace

extern "C" fp_status fp_batch_last_times(double* capture_ms, double* instantiate_ms, double* run_ms) {
    if (capture_ms) *capture_ms = g_batch_times.capture_ms;
    if (instantiate_ms) *instantiate_ms = g_batch_times.instantiate_ms;
    if (run_ms) *run_ms = g_batch_times.run_ms;
    return FP_OK;
}

namespace {
// library-owned streams for the jobs of a batch (0 .. 63) and a graph-capture origin (64), per
// device, created on first use
std::vector<std::pair<int, cudaStream_t>> g_job_streams;
cudaStream_t job_stream(uint32_t j) {
    int dev = 0;
    check(cudaGetDevice(&dev), "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_aux_mu);
    uint32_t have = 0;
    for (auto& e : g_job_streams)
        if (e.first == dev && have++ == j % 65) return e.second;
    while (have <= j % 65) {
        cudaStream_t st;
        check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate");
        g_job_streams.push_back({dev, st});
        if (have++ == j % 65) return st;
    }
    return nullptr;
}
}  // namespace

extern "C" {

fp_status vc_prove_all_batch(uint32_t njobs, const fp_job* jobs, int use_graph, void* stream, fp_proofs** outs) {
    if (!jobs || !outs) return njobs ? FP_EINVAL : FP_OK;
    g_batch_times = BatchTimes{};
    const auto t_start = std::chrono::steady_clock::now();
    auto ms_since = [](std::chrono::steady_clock::time_point a) {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - a).count();
    };
    for (uint32_t j = 0; j < njobs; j++) {
        const fp_commit* cm = jobs[j].cm;
        if (!cm || jobs[j].b < 1 || jobs[j].b > cm->pp->R) return FP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        std::vector<fp_proofs*> res(njobs, nullptr);
        std::vector<cudaStream_t> js(njobs);
        for (uint32_t j = 0; j < njobs; j++) js[j] = job_stream(j % 64);
        for (uint32_t j = 0; j < njobs; j++) (void)streams(js[j]);    // internal sets exist before capture
        bool capturing = false;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const cudaStream_t launch = s;
        if (use_graph) s = job_stream(64);            // capture origin: a library stream (the legacy
                                                      // default stream cannot be captured)
        try {
            if (use_graph) {
                check(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
                capturing = true;
            }
            cudaEvent_t fork = new_event();
            check(cudaEventRecord(fork, s), "event");
            for (uint32_t j = 0; j < njobs; j++) check(cudaStreamWaitEvent(js[j], fork, 0), "wait");
            for (uint32_t j = 0; j < njobs; j++) {
                const fp_commit* cm = jobs[j].cm;
                const uint32_t K = (cm->pp->R + jobs[j].b - 1) / jobs[j].b;
                res[j] = prove_impl(cm->pp, cm, jobs[j].b, 0, K, js[j], !use_graph);
            }
            for (uint32_t j = 0; j < njobs; j++) {
                cudaEvent_t e = new_event();
                check(cudaEventRecord(e, js[j]), "event");
                check(cudaStreamWaitEvent(s, e, 0), "join");
                cudaEventDestroy(e);
            }
            cudaEventDestroy(fork);
            if (use_graph) {
                capturing = false;
                check(cudaStreamEndCapture(s, &graph), "cudaStreamEndCapture");
                g_batch_times.capture_ms = ms_since(t_start);
                const auto t_inst = std::chrono::steady_clock::now();
                check(cudaGraphInstantiate(&exec, graph, 0), "cudaGraphInstantiate");
                g_batch_times.instantiate_ms = ms_since(t_inst);
                s = launch;
                for (uint32_t j = 0; j < njobs; j++)
                    if (jobs[j].cm->done) check(cudaStreamWaitEvent(s, jobs[j].cm->done, 0), "wait");
                const auto t_run = std::chrono::steady_clock::now();
                check(cudaGraphLaunch(exec, s), "cudaGraphLaunch");
                check(cudaStreamSynchronize(s), "vc_prove_all_batch");
                g_batch_times.run_ms = ms_since(t_run);
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                exec = nullptr;
                graph = nullptr;
                for (uint32_t j = 0; j < njobs; j++) {       // uses of the commitments, after the graph
                    const fp_commit* cm = jobs[j].cm;
                    cudaEvent_t used = new_event();
                    check(cudaEventRecord(used, s), "event");
                    std::lock_guard<std::mutex> lk(cm->mu);
                    cm->uses.push_back(used);
                }
                for (uint32_t j = 0; j < njobs; j++) res[j]->stream = s;
            }
        } catch (...) {
            if (capturing) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(s, &g);
                if (g) cudaGraphDestroy(g);
            }
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
            cudaStreamSynchronize(s);
            for (fp_proofs* p : res) fp_proofs_free(p);
            throw;
        }
        for (uint32_t j = 0; j < njobs; j++) outs[j] = res[j];
        return FP_OK;
    });
}

fp_status vc_verify(const fp_pp* pp, const uint8_t* C, uint32_t b, uint64_t i, const uint64_t m_i[4],
                    const uint8_t* proof, size_t len, void* stream) {
    if (!pp || !C || !m_i || !proof) return FP_EINVAL;
    if (b < 1 || b > pp->R || i >= (uint64_t)pp->R * pp->M) return FP_EINVAL;
    if (len != vc_proof_len(pp, b, i)) return FP_EVERIFY;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        const uint32_t k = (uint32_t)(i / pp->M) / b, lo = k * b, nk = std::min(b, pp->R - lo);
        const int lr = (int)pp->log_r, lc = (int)pp->log_c;
        // proof | C | m_i (32 bytes big-endian), one host-to-device copy
        std::vector<uint8_t> host(len + GT_SER + 32);
        memcpy(host.data(), proof, len);
        memcpy(host.data() + len, C, GT_SER);
        for (int w = 0; w < 4; w++)
            for (int q = 0; q < 8; q++) host[len + GT_SER + 8 * (3 - w) + q] = (uint8_t)(m_i[w] >> (56 - 8 * q));
        void *dbuf = nullptr, *scr = nullptr, *res = nullptr;
        uint32_t hres = 1;
        try {
            dbuf = dalloc(host.size(), s);
            scr = dalloc(verify_scratch_bytes(b, lr, lc), s);
            res = dalloc(sizeof(uint32_t), s);
            check(cudaMemcpyAsync(dbuf, host.data(), host.size(), cudaMemcpyHostToDevice, s), "H2D proof");
            const uint8_t* d = (const uint8_t*)dbuf;
            verify_one(d, d + len, d + len + GT_SER, nk, lr, lc, b, i, pp->M, k, lo, pp->g1beta, pp->g2tau, scr,
                       (uint32_t*)res, s);
            check_launch("vc_verify kernels");
            check(cudaMemcpyAsync(&hres, res, sizeof hres, cudaMemcpyDeviceToHost, s), "D2H result");
            dfree(dbuf, s); dfree(scr, s); dfree(res, s);
            check(cudaStreamSynchronize(s), "vc_verify");
        } catch (...) {
            cudaStreamSynchronize(s);
            dfree(dbuf, s); dfree(scr, s); dfree(res, s);
            throw;
        }
        return hres ? FP_EVERIFY : FP_OK;
    });
}

fp_status vc_verify_all(const fp_pp* pp, const uint8_t* C, const uint64_t* m, int on_device, const fp_proofs* pf,
                        int flags, void* stream, uint8_t* ok, uint64_t* n_ok) {
    if (!pp || !C || !m || !pf || pf->pp != pp || (flags & ~1) || !pf->step2 || pf->nopen != pf->L.K) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        const ProofLayout& L = pf->L;
        const uint64_t N = (uint64_t)L.R * L.M;
        void *dC = nullptr, *dm = nullptr, *scr = nullptr;
        cudaEvent_t ready = nullptr;
        try {
            // the proof pieces are written on the handle's stream
            check(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming), "cudaEventCreate");
            check(cudaEventRecord(ready, pf->stream), "cudaEventRecord");
            check(cudaStreamWaitEvent(s, ready, 0), "cudaStreamWaitEvent");
            dC = dalloc(GT_SER, s);
            check(cudaMemcpyAsync(dC, C, GT_SER, cudaMemcpyHostToDevice, s), "H2D C");
            const void* md = m;
            if (!on_device) {
                dm = dalloc(N * 32, s);
                check(cudaMemcpyAsync(dm, m, N * 32, cudaMemcpyHostToDevice, s), "H2D m");
                md = dm;
            }
            scr = dalloc(verify_all_scratch_bytes(L), s);
            const uint64_t good = verify_all(L, dC, md, pf->rows_ser, pf->blocks, pf->row_tree, pf->top_tree, pf->D_ser,
                                             pf->g, pf->pst_ser, pp->g1beta, pp->g2tau, flags & 1, scr, ok, s);
            check_launch("vc_verify_all kernels");
            dfree(dC, s); dfree(dm, s); dfree(scr, s);
            check(cudaStreamSynchronize(s), "vc_verify_all");
            cudaEventDestroy(ready);
            if (n_ok) *n_ok = good;
        } catch (...) {
            cudaStreamSynchronize(s);
            dfree(dC, s); dfree(dm, s); dfree(scr, s);
            if (ready) cudaEventDestroy(ready);
            throw;
        }
        return FP_OK;
    });
}

size_t vc_eval_proof_len(const fp_pp* pp) {
    if (!pp) return 0;
    return 32 + G1_SER + bopen_len(pp->log_r) + G1_SER * (size_t)pp->log_c;
}

fp_status vc_eval_prove(const fp_pp* pp, const fp_commit* cm, const uint8_t* r, void* stream, uint8_t* out,
                        size_t cap, size_t* len) {
    if (!pp || !cm || !r || !len || cm->pp != pp) return FP_EINVAL;
    const size_t need = vc_eval_proof_len(pp);
    *len = need;
    if (!out) return FP_OK;
    if (cap < need) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        const uint32_t R = pp->R, M = pp->M;
        const int lr = (int)pp->log_r, lc = (int)pp->log_c, ln = (int)pp->log_n;
        const size_t blen = bopen_len(pp->log_r);
        const uint64_t half = M / 2 ? M / 2 : 1;
        const MsmShape sh = msm_shape(R, 1, R, fp_msm_window(R, 1));
        std::vector<void*> tmp;
        auto T = [&](size_t bytes) { void* p = dalloc(bytes, s); tmp.push_back(p); return p; };
        uint32_t herr = 0;
        try {
            if (cm->done) check(cudaStreamWaitEvent(s, cm->done, 0), "wait");
            uint8_t* proof = (uint8_t*)T(need);                 // y | C_F | pi_FC | pi_PST
            void* r_be = T(32 * (size_t)ln);
            void* r_mont = T((size_t)ln * FR_BYTES);
            uint32_t* err = (uint32_t*)T(4);
            void* Tm = T((size_t)R * FR_BYTES);
            void* Tc = T((size_t)R * FR_BYTES);
            void* F = T((size_t)M * FR_BYTES);
            void* q = T((size_t)M * FR_BYTES);
            void* tab = T(2 * (size_t)R * G1A_BYTES);
            void* mscr = T(msm_scratch_bytes(sh));
            void* r0 = T(FR_BYTES);
            void* terms = T((size_t)(lc ? lc : 1) * half * G1J_BYTES);
            void* terms2 = T((half / 2 + 1) * G1J_BYTES);
            const Step1Bufs B = step1_bufs(pp, 1, T);
            const bool la = lookahead_on((int)pp->log_r);
            const LaBufs L = la ? la_bufs(pp, 1, T) : LaBufs{};
            const Streams st = streams(s);
            cudaStream_t s1 = st.hi, s3 = st.sp;
            cudaEvent_t ev_fork = new_event(), ev_bvec = new_event(), ev_join = new_event();
            check(cudaEventRecord(ev_fork, s), "event");
            check(cudaStreamWaitEvent(s1, ev_fork, 0), "wait");
            check(cudaMemsetAsync(err, 0, 4, s1), "memset");
            check(cudaMemcpyAsync(r_be, r, 32 * (size_t)ln, cudaMemcpyHostToDevice, s1), "H2D r");
            eval_point(r_be, ln, r_mont, err, s1);
            eval_weights(r_mont, lr, lc, Tm, Tc, s1);
            // step 1: C_F = sum_j T_j C_j over the row commitments (and their GLV partners)
            check(cudaMemcpyAsync(tab, cm->rows, (size_t)R * G1A_BYTES, cudaMemcpyDeviceToDevice, s1), "D2D");
            msm_bases_endo(tab, R, s1);
            msm_g1(tab, Tc, sh, mscr, nullptr, proof + 32, s1);
            // step 2: FC.BOpen of <C, T> with t = 1 through the Step-1 round chain (one block of R rows)
            step1_init(cm->rows, pp->g2pow, 1, R, B.A, B.v, B.bvec, s1);
            eval_bvec(cm->C_ser, r_be, ln, proof + 32, Tm, R, r0, B.bvec, s1);
            check(cudaEventRecord(ev_bvec, s1), "event");
            check(cudaStreamWaitEvent(s3, ev_bvec, 0), "wait");
            if (la) step1_rounds_la(pp, 0, 1, R, B, L, proof + 128, blen, s1, s3, st.pre, st.la, st.fold);
            else step1_rounds(pp, 0, 1, R, B, proof + 128, blen, s1, s3, st.pre);
            // step 3: PST.Eval of F = sum_j T_j f_j at r_R
            eval_ftable(cm->m_mont, Tm, R, M, F, s1);
            eval_pst_fold(F, r_mont, lc, q, proof, s1);
            if (lc) {
                check(cudaMemsetAsync(terms, 0, (size_t)lc * half * G1J_BYTES, s1), "memset");
                eval_pst_terms(q, pp->lam, M, terms, s1);
                for (int t = 0; t < lc; t++) {
                    void* lvl = (uint8_t*)terms + (size_t)t * half * G1J_BYTES;
                    void* res = reduce_pairs(lvl, terms2, half, 1, g1_pair_reduce, s1);
                    g1j_to_affine(res, nullptr, proof + 128 + blen + G1_SER * (size_t)(lc - 1 - t), G1_SER, 1, s1);
                }
            }
            check_launch("vc_eval_prove kernels");
            check(cudaMemcpyAsync(out, proof, need, cudaMemcpyDeviceToHost, s1), "D2H proof");
            check(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s1), "D2H err");
            check(cudaEventRecord(ev_join, s1), "event");
            check(cudaStreamWaitEvent(s, ev_join, 0), "join");
            for (void* p : tmp) cudaFreeAsync(p, s);
            tmp.clear();
            cudaEventDestroy(ev_fork); cudaEventDestroy(ev_bvec); cudaEventDestroy(ev_join);
            check(cudaStreamSynchronize(s), "vc_eval_prove");
        } catch (...) {
            for (void* p : tmp) cudaFreeAsync(p, s);
            cudaStreamSynchronize(s);
            throw;
        }
        return herr ? FP_ERANGE : FP_OK;
    });
}

fp_status vc_eval_verify(const fp_pp* pp, const uint8_t* C, const uint8_t* r, const uint8_t* proof, size_t len,
                         void* stream) {
    if (!pp || !C || !r || !proof) return FP_EINVAL;
    if (len != vc_eval_proof_len(pp)) return FP_EVERIFY;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        const int ln = (int)pp->log_n;
        // proof | C | r, one host-to-device copy
        std::vector<uint8_t> host(len + GT_SER + 32 * (size_t)ln);
        memcpy(host.data(), proof, len);
        memcpy(host.data() + len, C, GT_SER);
        memcpy(host.data() + len + GT_SER, r, 32 * (size_t)ln);
        void *dbuf = nullptr, *scr = nullptr, *res = nullptr;
        uint32_t hres = 1;
        try {
            dbuf = dalloc(host.size(), s);
            scr = dalloc(verify_eval_scratch_bytes(pp->R, (int)pp->log_r, (int)pp->log_c, ln), s);
            res = dalloc(sizeof(uint32_t), s);
            check(cudaMemcpyAsync(dbuf, host.data(), host.size(), cudaMemcpyHostToDevice, s), "H2D");
            const uint8_t* d = (const uint8_t*)dbuf;
            verify_eval(d, d + len, d + len + GT_SER, ln, (int)pp->log_r, (int)pp->log_c, pp->R, pp->g1beta,
                        pp->g2tau, scr, (uint32_t*)res, s);
            check_launch("vc_eval_verify kernels");
            check(cudaMemcpyAsync(&hres, res, sizeof hres, cudaMemcpyDeviceToHost, s), "D2H result");
            dfree(dbuf, s); dfree(scr, s); dfree(res, s);
            check(cudaStreamSynchronize(s), "vc_eval_verify");
        } catch (...) {
            cudaStreamSynchronize(s);
            dfree(dbuf, s); dfree(scr, s); dfree(res, s);
            throw;
        }
        return hres ? FP_EVERIFY : FP_OK;
    });
}

fp_status vc_open_segments(const fp_pp* pp, const fp_commit* cm, uint32_t b, uint32_t k0, uint32_t nblocks,
                           void* stream, fp_proofs** out) {
    if (!pp || !cm || !out || cm->pp != pp) return FP_EINVAL;
    if (b < 1 || b > pp->R) return FP_EINVAL;
    const uint32_t K = (pp->R + b - 1) / b;
    if (k0 >= K) return FP_EINVAL;
    if (nblocks == 0) nblocks = K - k0;
    if (nblocks > K - k0) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        *out = prove_impl(pp, cm, b, k0, nblocks, (cudaStream_t)stream, true, false);
        return FP_OK;
    });
}

size_t vc_segment_proof_len(const fp_pp* pp, uint32_t b, uint32_t j) {
    if (!pp || b < 1 || b > pp->R || j >= pp->R) return 0;
    const uint32_t lo = (j / b) * b, nk = std::min(b, pp->R - lo);
    return (size_t)nk * G1_SER + bopen_len(pp->log_r);
}

fp_status vc_segment_proof_get(const fp_proofs* pf, uint32_t j, uint8_t* out, size_t cap, size_t* len) {
    if (!pf || !len) return FP_EINVAL;
    const ProofLayout& L = pf->L;
    if (j >= L.R) return FP_EINVAL;
    const uint32_t k = j / L.b, lo = k * L.b, nk = std::min(L.b, L.R - lo);
    if (k < pf->k0 || k >= pf->k0 + pf->nopen) return FP_EINVAL;
    const size_t need = (size_t)nk * G1_SER + L.bopen_len;
    *len = need;
    if (!out) return FP_OK;
    if (cap < need) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        cudaStream_t s = pf->stream;
        check(cudaMemcpyAsync(out, (const uint8_t*)pf->rows_ser + (size_t)lo * G1_SER, (size_t)nk * G1_SER,
                              cudaMemcpyDeviceToHost, s), "D2H block");
        check(cudaMemcpyAsync(out + (size_t)nk * G1_SER, (const uint8_t*)pf->blocks + (size_t)k * L.bopen_len,
                              L.bopen_len, cudaMemcpyDeviceToHost, s), "D2H pi_Ck");
        check(cudaStreamSynchronize(s), "vc_segment_proof_get");
        return FP_OK;
    });
}

fp_status vc_verify_segment(const fp_pp* pp, const uint8_t* C, uint32_t b, uint32_t j, const uint64_t* m_j,
                            const uint8_t* proof, size_t len, void* stream) {
    if (!pp || !C || !m_j || !proof) return FP_EINVAL;
    if (b < 1 || b > pp->R || j >= pp->R) return FP_EINVAL;
    if (len != vc_segment_proof_len(pp, b, j)) return FP_EVERIFY;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        const uint32_t M = pp->M, k = j / b, lo = k * b, nk = std::min(b, pp->R - lo);
        const int lr = (int)pp->log_r;
        const MsmShape sh = msm_shape(M, 1, M, fp_msm_window(M, 1));
        // proof | C | m_j, one host-to-device copy
        const size_t mbytes = (size_t)M * 32;
        std::vector<uint8_t> host(len + GT_SER + mbytes);
        memcpy(host.data(), proof, len);
        memcpy(host.data() + len, C, GT_SER);
        memcpy(host.data() + len + GT_SER, m_j, mbytes);
        void *dbuf = nullptr, *vscr = nullptr, *mscr = nullptr, *mc = nullptr, *mm = nullptr, *cj = nullptr,
             *out = nullptr;
        uint32_t hout[2 + 24] = {};
        try {
            dbuf = dalloc(host.size(), s);
            vscr = dalloc(verify_block_scratch_bytes(b, lr), s);
            mscr = dalloc(msm_scratch_bytes(sh), s);
            mc = dalloc(mbytes, s);
            mm = dalloc(mbytes, s);
            cj = dalloc(G1A_BYTES, s);
            out = dalloc(sizeof hout, s);         // [block result, range error, C_j serialised (96 B)]
            check(cudaMemsetAsync(out, 0, sizeof hout, s), "memset");
            check(cudaMemcpyAsync(dbuf, host.data(), host.size(), cudaMemcpyHostToDevice, s), "H2D");
            const uint8_t* d = (const uint8_t*)dbuf;
            uint32_t* o = (uint32_t*)out;
            load_vector(d + len + GT_SER, M, mc, mm, o + 1, s);
            msm_g1(pp->lam_tab, mc, sh, mscr, cj, o + 2, s);       // C_j from m_j (VC.Commit's row MSM)
            verify_block(d, d + (size_t)nk * G1_SER, d + len, nk, lr, b, k, lo, pp->g1beta, vscr, o, s);
            check_launch("vc_verify_segment kernels");
            check(cudaMemcpyAsync(hout, out, sizeof hout, cudaMemcpyDeviceToHost, s), "D2H");
            dfree(dbuf, s); dfree(vscr, s); dfree(mscr, s); dfree(mc, s); dfree(mm, s); dfree(cj, s); dfree(out, s);
            check(cudaStreamSynchronize(s), "vc_verify_segment");
        } catch (...) {
            cudaStreamSynchronize(s);
            dfree(dbuf, s); dfree(vscr, s); dfree(mscr, s); dfree(mc, s); dfree(mm, s); dfree(cj, s); dfree(out, s);
            throw;
        }
        const bool same = memcmp(hout + 2, proof + (size_t)(j - lo) * G1_SER, G1_SER) == 0;
        return (hout[0] == 0 && hout[1] == 0 && same) ? FP_OK : FP_EVERIFY;
    });
}

fp_status vc_prove_one(const fp_pp* pp, const fp_commit* cm, uint32_t b, uint64_t i, void* stream, uint8_t* out,
                       size_t cap, size_t* len) {
    if (!pp || !cm || !len || cm->pp != pp) return FP_EINVAL;
    if (b < 1 || b > pp->R || i >= (uint64_t)pp->R * pp->M) return FP_EINVAL;
    const size_t need = vc_proof_len(pp, b, i);
    *len = need;
    if (!out) return FP_OK;
    if (cap < need) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        const uint32_t k = (uint32_t)(i / pp->M) / b;
        fp_proofs* pf = prove_impl(pp, cm, b, k, 1, (cudaStream_t)stream);
        const fp_status st = vc_proof_get(pf, i, out, cap, len);
        fp_proofs_free(pf);
        return st;
    });
}

size_t vc_proof_len(const fp_pp* pp, uint32_t b, uint64_t i) {
    if (!pp || b < 1 || b > pp->R || i >= (uint64_t)pp->R * pp->M) return 0;
    ProofLayout L{pp->R, pp->M, b, (pp->R + b - 1) / b, (int)pp->log_n, (int)pp->log_r, (int)pp->log_c,
                  bopen_len(pp->log_r)};
    return proof_len(L, i);
}

fp_status vc_proofs_export(const fp_proofs* pf, uint64_t i0, uint64_t count, uint8_t* out, size_t cap, size_t* len) {
    if (!pf || !len || !pf->step2) return FP_EINVAL;
    const ProofLayout& L = pf->L;
    const uint64_t N = (uint64_t)L.R * L.M;
    if (count == 0 || i0 >= N || count > N - i0) return FP_EINVAL;
    const uint64_t ka = (i0 / L.M) / L.b, kb = ((i0 + count - 1) / L.M) / L.b;
    if (ka < pf->k0 || kb >= (uint64_t)pf->k0 + pf->nopen) return FP_EINVAL;
    size_t total = 0;
    for (uint64_t q = 0; q < count; q++) total += proof_len(L, i0 + q);
    *len = total;
    if (!out) return FP_OK;
    if (cap < total) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        cudaStream_t s = pf->stream;
        void* d = dalloc(total, s);
        assemble(L, pf->rows_ser, pf->blocks, pf->row_tree, pf->top_tree, pf->D_ser, pf->g, pf->pst_ser, i0, count, d,
                 s);
        check_launch("assemble");
        check(cudaMemcpyAsync(out, d, total, cudaMemcpyDeviceToHost, s), "D2H proofs");
        dfree(d, s);
        check(cudaStreamSynchronize(s), "vc_proofs_export");
        return FP_OK;
    });
}

fp_status vc_proof_get(const fp_proofs* pf, uint64_t i, uint8_t* out, size_t cap, size_t* len) {
    return vc_proofs_export(pf, i, 1, out, cap, len);
}

fp_status vc_proofs_state(const fp_proofs* pf, uint8_t* out, size_t cap, size_t* len) {
    if (!pf || !len || !pf->step2) return FP_EINVAL;
    const ProofLayout& L = pf->L;
    const uint64_t ng = (2 * (uint64_t)L.R - 1) * L.M;
    const size_t parts[7] = {(size_t)L.K * L.bopen_len, (size_t)L.R * (2 * L.M - 1) * DIGEST,
                             (2 * (size_t)L.R - 1) * DIGEST, (size_t)L.R * 32, (2 * (size_t)L.R - 1) * G1_SER,
                             ng * 32, ((size_t)L.M - 1) * G1_SER};
    size_t total = 0;
    for (size_t p : parts) total += p;
    *len = total;
    if (!out) return FP_OK;
    if (cap < total) return FP_EINVAL;
    return guarded([&]() -> fp_status {
        cudaStream_t s = pf->stream;
        // r_j and the fold tables leave in the exchanged encoding (canonical big-endian)
        void* d = dalloc(parts[3] + parts[5], s);
        fr_serialize(pf->rj, L.R, d, s);
        fr_serialize(pf->g, ng, (uint8_t*)d + parts[3], s);
        check_launch("vc_proofs_state");
        const void* src[7] = {pf->blocks, pf->row_tree, pf->top_tree, d, pf->D_ser, (uint8_t*)d + parts[3],
                              pf->pst_ser};
        size_t off = 0;
        for (int q = 0; q < 7; q++) {
            check(cudaMemcpyAsync(out + off, src[q], parts[q], cudaMemcpyDeviceToHost, s), "D2H state");
            off += parts[q];
        }
        dfree(d, s);
        check(cudaStreamSynchronize(s), "vc_proofs_state");
        return FP_OK;
    });
}

fp_status vc_proofs_step2_parts(const fp_proofs* pf, uint8_t* root, uint8_t* rj, uint8_t* gstar, uint8_t* dstar) {
    if (!pf || !pf->step2) return FP_EINVAL;
    const ProofLayout& L = pf->L;
    return guarded([&]() -> fp_status {
        cudaStream_t s = pf->stream;
        void* d = dalloc(((size_t)L.R + L.M) * 32, s);
        fr_serialize(pf->rj, L.R, d, s);
        step2_gstar_ser(pf->g, L.R, L.M, (uint8_t*)d + (size_t)L.R * 32, s);
        check_launch("step2 parts");
        if (root)
            check(cudaMemcpyAsync(root, (uint8_t*)pf->top_tree + (2 * (size_t)L.R - 2) * DIGEST, 32,
                                  cudaMemcpyDeviceToHost, s), "D2H");
        if (rj) check(cudaMemcpyAsync(rj, d, (size_t)L.R * 32, cudaMemcpyDeviceToHost, s), "D2H");
        if (gstar) check(cudaMemcpyAsync(gstar, (uint8_t*)d + (size_t)L.R * 32, (size_t)L.M * 32,
                                         cudaMemcpyDeviceToHost, s), "D2H");
        if (dstar)
            check(cudaMemcpyAsync(dstar, (uint8_t*)pf->D_ser + (2 * (size_t)L.R - 2) * G1_SER, G1_SER,
                                  cudaMemcpyDeviceToHost, s), "D2H");
        dfree(d, s);
        check(cudaStreamSynchronize(s), "vc_proofs_step2_parts");
        return FP_OK;
    });
}

/* ---------------------------------------------------------------- G1 multi-scalar multiplication */

fp_status fp_g1_bases_from_scalars(const uint64_t* s_limbs, uint64_t n, int on_device, void* stream,
                                   fp_g1_bases** out) {
    if (!out || (!s_limbs && n) || n >= (1ull << 30)) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        fp_g1_bases* P = new fp_g1_bases{n};
        void* src = nullptr;
        try {
            P->tab = dalloc(2 * n * G1A_BYTES, s);
            const void* sc = s_limbs;
            if (!on_device && n) {
                src = dalloc(n * FR_BYTES, s);
                check(cudaMemcpyAsync(src, s_limbs, n * FR_BYTES, cudaMemcpyHostToDevice, s), "H2D s");
                sc = src;
            }
            if (n) g1_gen_mul(sc, (uint32_t)n, P->tab, s);
            msm_bases_endo(P->tab, n, s);
            check_launch("fp_g1_bases_from_scalars");
            dfree(src, s);
            check(cudaStreamSynchronize(s), "fp_g1_bases_from_scalars");
        } catch (...) {
            cudaStreamSynchronize(s);
            fp_g1_bases_free(P);
            throw;
        }
        *out = P;
        return FP_OK;
    });
}

fp_status fp_g1_bases_load(const uint8_t* pts, uint64_t n, int on_device, void* stream, fp_g1_bases** out) {
    if (!out || (!pts && n) || n >= (1ull << 30)) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        fp_g1_bases* P = new fp_g1_bases{n};
        void* src = nullptr;
        uint32_t* err = nullptr;
        uint32_t herr = 0;
        try {
            P->tab = dalloc(2 * n * G1A_BYTES, s);
            err = (uint32_t*)dalloc(sizeof(uint32_t), s);
            check(cudaMemsetAsync(err, 0, sizeof(uint32_t), s), "memset");
            const void* be = pts;
            if (!on_device && n) {
                src = dalloc(n * G1_SER, s);
                check(cudaMemcpyAsync(src, pts, n * G1_SER, cudaMemcpyHostToDevice, s), "H2D points");
                be = src;
            }
            msm_bases_load(be, n, P->tab, err, s);
            check_launch("fp_g1_bases_load");
            check(cudaMemcpyAsync(&herr, err, sizeof herr, cudaMemcpyDeviceToHost, s), "D2H err");
            dfree(src, s);
            void* e = err;
            dfree(e, s);
            check(cudaStreamSynchronize(s), "fp_g1_bases_load");
        } catch (...) {
            cudaStreamSynchronize(s);
            fp_g1_bases_free(P);
            throw;
        }
        if (herr) {
            fp_g1_bases_free(P);
            return FP_EINVAL;
        }
        *out = P;
        return FP_OK;
    });
}

uint64_t fp_g1_bases_count(const fp_g1_bases* P) { return P ? P->n : 0; }

}  // extern "C"

namespace {
// windows chosen by fp_msm_autotune, per (terms, batches)
std::mutex g_tune_mu;
std::vector<std::pair<std::pair<uint64_t, uint32_t>, int>> g_tuned;

int tuned_window(uint64_t n, uint32_t nbatch) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (auto& e : g_tuned)
        if (e.first.first == n && e.first.second == nbatch) return e.second;
    return 0;
}

bool msm_shape_ok(const MsmShape& sh) {
    return sh.entries_max() <= 0xffffffffull && sh.nkeys() <= 0xffffffffull;
}

// enqueue one MSM; the scalars and the serialised output are device pointers
void msm_enqueue(const fp_g1_bases* P, const void* k_dev, const MsmShape& sh, void* out_ser, cudaStream_t s) {
    void* scratch = dalloc(msm_scratch_bytes(sh), s);
    msm_g1(P->tab, k_dev, sh, scratch, nullptr, out_ser, s);
    check_launch("fp_msm_g1");
    dfree(scratch, s);
}
}  // namespace

extern "C" {

int fp_msm_window_g2(uint64_t n, uint32_t nbatch) { return msm_window_model(n, nbatch, 4, 65, 3.0); }

int fp_msm_window(uint64_t n, uint32_t nbatch) {
    const int t = tuned_window(n, nbatch);
    return t ? t : msm_window_model(n, nbatch);
}

fp_status fp_msm_g1(const fp_g1_bases* P, const uint64_t* k, uint64_t n, uint32_t nbatch, int on_device,
                    int window, void* stream, uint8_t* out) {
    if (!P || !out || (!k && n && nbatch) || (n && !P->n)) return FP_EINVAL;
    if (window != 0 && (window < 4 || window > 16)) return FP_EINVAL;
    if (!nbatch) return FP_OK;
    const int c = window ? window : fp_msm_window(n, nbatch);
    const MsmShape sh = msm_shape(n, nbatch, P->n ? P->n : 1, c);
    if (!msm_shape_ok(sh)) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        void *kd = nullptr, *od = nullptr;
        try {
            const void* kp = k;
            void* op = out;
            if (!on_device) {
                kd = dalloc(n * nbatch * FR_BYTES, s);
                if (n) check(cudaMemcpyAsync(kd, k, n * nbatch * FR_BYTES, cudaMemcpyHostToDevice, s), "H2D k");
                od = dalloc((size_t)nbatch * G1_SER, s);
                kp = kd;
                op = od;
            }
            msm_enqueue(P, kp, sh, op, s);
            if (!on_device) {
                check(cudaMemcpyAsync(out, od, (size_t)nbatch * G1_SER, cudaMemcpyDeviceToHost, s), "D2H msm");
                dfree(kd, s);
                dfree(od, s);
                check(cudaStreamSynchronize(s), "fp_msm_g1");
            }
        } catch (...) {
            cudaStreamSynchronize(s);
            dfree(kd, s);
            dfree(od, s);
            throw;
        }
        return FP_OK;
    });
}

fp_status fp_msm_autotune(const fp_g1_bases* P, const uint64_t* k_dev, uint64_t n, uint32_t nbatch, void* stream,
                          int* window, double* best_ms) {
    if (!P || !window || !k_dev || !n || !nbatch || !P->n) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return guarded([&]() -> fp_status {
        const int c0 = msm_window_model(n, nbatch);
        void* od = dalloc((size_t)nbatch * G1_SER, s);
        cudaEvent_t e0, e1;
        check(cudaEventCreate(&e0), "cudaEventCreate");
        check(cudaEventCreate(&e1), "cudaEventCreate");
        int best = c0;
        float bt = 1e30f;
        for (int c = std::max(4, c0 - 3); c <= std::min(16, c0 + 3); c++) {
            const MsmShape sh = msm_shape(n, nbatch, P->n, c);
            if (!msm_shape_ok(sh)) continue;
            msm_enqueue(P, k_dev, sh, od, s);            // warm-up (allocation pool, caches)
            check(cudaEventRecord(e0, s), "cudaEventRecord");
            msm_enqueue(P, k_dev, sh, od, s);
            check(cudaEventRecord(e1, s), "cudaEventRecord");
            check(cudaEventSynchronize(e1), "cudaEventSynchronize");
            float ms = 0;
            check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            if (ms < bt) {
                bt = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dfree(od, s);
        check(cudaStreamSynchronize(s), "fp_msm_autotune");
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            bool found = false;
            for (auto& e : g_tuned)
                if (e.first.first == n && e.first.second == nbatch) { e.second = best; found = true; }
            if (!found) g_tuned.push_back({{n, nbatch}, best});
        }
        *window = best;
        if (best_ms) *best_ms = bt;
        return FP_OK;
    });
}

void fp_g1_bases_free(fp_g1_bases* P) {
    if (!P) return;
    cudaDeviceSynchronize();
    cudaFree(P->tab);
    delete P;
}


void fp_pp_free(fp_pp* pp) {
    if (!pp) return;
    cudaDeviceSynchronize();
    cudaFree(pp->lam_tab);
    cudaFree(pp->lam_comb);
    cudaFree(pp->g2w_tab);
    if (!pp->parent) {
        cudaFree(pp->lam); cudaFree(pp->g1beta); cudaFree(pp->g2pow); cudaFree(pp->g2tau); cudaFree(pp->g2comb);
    }
    delete pp;
}
void fp_commit_free(fp_commit* cm) {
    if (!cm) return;
    // stream-ordered release on an internal stream, after the commit's own work and every
    // recorded use of the handle
    cudaStream_t fs = nullptr;
    try {
        fs = streams(cm->stream).lo;
    } catch (...) {
        fs = nullptr;
    }
    if (!fs) {
        cudaDeviceSynchronize();
    } else {
        if (cm->done) cudaStreamWaitEvent(fs, cm->done, 0);
        std::lock_guard<std::mutex> lk(cm->mu);
        for (cudaEvent_t e : cm->uses) cudaStreamWaitEvent(fs, e, 0);
    }
    for (void* p : {cm->m_canon, cm->m_mont, cm->rows, cm->rows_ser, cm->C, cm->C_ser, (void*)cm->err})
        if (p) cudaFreeAsync(p, fs);
    if (cm->done) cudaEventDestroy(cm->done);
    if (cm->rows_done) cudaEventDestroy(cm->rows_done);
    for (cudaEvent_t e : cm->uses) cudaEventDestroy(e);
    delete cm;
}
void fp_proofs_free(fp_proofs* pf) {
    if (!pf) return;
    // every use of the handle is ordered on its stream (creation joins back to it, getters
    // synchronise it): release stream-ordered there
    for (void* p : {pf->rows_ser, pf->blocks, pf->row_tree, pf->top_tree, pf->rj, pf->g, pf->D, pf->D_ser,
                    pf->pst_ser})
        if (p) cudaFreeAsync(p, pf->stream);
    delete pf;
}

}  // extern "C"
