// Host-side launchers of the FlexProofs kernels.  Plain C++ (no device types): every buffer is
// passed as an untyped device pointer whose element layout is fixed by the byte sizes below.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "msm.h"

namespace fpk {

// Every kernel launch goes through FP_KERNEL: it counts the launch and, while profiling is
// enabled, brackets it with CUDA events on the launching stream (per-kernel totals).
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);
#define FP_KERNEL(name, stream, ...) \
    do {                             \
        fpk::prof_begin(name, stream); \
        __VA_ARGS__;                 \
        fpk::prof_end(stream);       \
    } while (0)

// Engine choice by size: the launchers pick a latency engine (one 128-thread block or one warp per
// pairing, final exponentiation or point) for few items and a throughput engine (one thread each)
// for many.  The limits are process-wide (fp_set_engine_limits); every decision reads them once, and
// every engine computes the same values, so a limit changes which kernels run, never the bytes.
struct EngineLimits {
    uint32_t miller_block_max = 1024;       // Step-1 Miller loops per launch: <= this, a block each
    uint32_t miller_warp_max = 16383;       //   <= this, a warp each; above, a thread each
    uint32_t miller_group_min = 1u << 18;   //   from this many (h >= 4), 4 pairs of a product per thread
    uint32_t commit_block_max = 1024;       // Commit's Miller loops: <= this, a block each
    uint32_t commit_warp_max = 16384;       //   <= this, a warp each; above, a thread each
    uint32_t fe_block_max = 256;            // final exponentiations per launch: <= this, a block each
    uint32_t fe_warp_max = 0xffffffffu;     //   <= this, a warp each; above, a thread each
    uint32_t pair_block_max = 2048;         // pairwise Fq12 products: <= this, a block each; above, a thread
    uint32_t fold_warp_max = 4096;          // fold points (beyond the split folds): <= this, a warp / 8 lanes
                                            //   per point; above, a thread per point
    uint32_t wterm_warp_max = 4096;         // W terms: <= this, a warp per term; above, a thread per term
    uint32_t msm_chunks = 1u << 17;         // MSM bucket pass: about this many chunks of the entry list
    uint32_t msm_segment_threads = 1u << 15;  // MSM bucket reduction: at most about this many segments
};
EngineLimits engine_limits();              // a snapshot of the current limits

constexpr size_t FR_BYTES = 32;     // fr: 8 x u32, Montgomery or canonical as documented
constexpr size_t G1A_BYTES = 96;    // affine G1, Montgomery, (0,0) = identity
constexpr size_t G1J_BYTES = 144;   // Jacobian G1
constexpr size_t G2A_BYTES = 192;   // affine G2
constexpr size_t G2J_BYTES = 288;   // Jacobian G2
constexpr size_t FQ12_BYTES = 576;  // Fq12 (Montgomery limbs, tower order)
constexpr size_t GT_SER = 576, G1_SER = 96, G2_SER = 192, DIGEST = 32;
constexpr size_t ROUND_BYTES = 2 * GT_SER + 2 * G1_SER;   // L_j.T, L_j.1, R_j.T, R_j.1

// ---- setup
void setup_trapdoor(uint64_t seed, int log_c, void* trap_fr, cudaStream_t s);
void setup_scalars(const void* trap_fr, int log_r, int log_c, void* lam_scal, void* pow_scal, void* tau_scal,
                   void* beta_scal, cudaStream_t s);
void g1_gen_mul(const void* scal_canon, uint32_t n, void* out_g1a, cudaStream_t s);
void g2_gen_mul(const void* scal_canon, uint32_t n, void* out_g2a, cudaStream_t s);

// ---- generic group helpers
void g1_pair_reduce(const void* in_g1j, void* out_g1j, uint64_t n_out, cudaStream_t s);
void g2_pair_reduce(const void* in_g2j, void* out_g2j, uint64_t n_out, cudaStream_t s);
// out[g] = sum of in[gs g .. gs g + gs - 1] (Jacobian; gs <= 32 on G1, <= 16 on G2), one block per
// sum on the lane-parallel group engines: few sums of many points, for latency
void g1_tree_reduce(const void* in_g1j, void* out_g1j, uint64_t n_in, uint32_t gs, cudaStream_t s);
void g2_tree_reduce(const void* in_g2j, void* out_g2j, uint64_t n_in, uint32_t gs, cudaStream_t s);
void fq12_pair_reduce(const void* in, void* out, uint64_t n_out, cudaStream_t s);
void g1j_to_affine(const void* in_g1j, void* out_g1a, void* ser_out, size_t ser_stride, uint64_t n, cudaStream_t s);
void g2j_to_affine(const void* in_g2j, void* out_g2a, void* ser_out, size_t ser_stride, uint64_t n, cudaStream_t s);
void g1a_serialize(const void* in_g1a, void* ser_out, size_t ser_stride, uint64_t n, cudaStream_t s);
void g2a_serialize(const void* in_g2a, void* ser_out, size_t ser_stride, uint64_t n, cudaStream_t s);

void fr_serialize(const void* fr_mont, uint64_t n, void* out, cudaStream_t s);

// ---- commit
void load_vector(const void* m_limbs, uint64_t n, void* m_canon, void* m_mont, uint32_t* err, cudaStream_t s);
// out[j] = ML(rows[j], g2pow[2 j])
void commit_miller(const void* rows_g1a, const void* g2pow, uint32_t R, void* out_fq12, cudaStream_t s);
void final_exp_group(const void* in_fq12, uint32_t n, void* out_fq12, void* ser, uint32_t per, size_t stride_a,
                     size_t stride_b, cudaStream_t s);

// ---- Step 1 (FC.BOpen for all blocks at once)
void step1_init(const void* rows_g1a, const void* g2pow, uint32_t K, uint32_t R, void* A, void* v, void* bvec,
                cudaStream_t s);
// blocks k0 .. k0 + K - 1 of size b (stored at local indices 0 .. K - 1); the statement digests go
// to hstmt (32 bytes per block), through scratch (stmt_hash_scratch_bytes) for the row trees
size_t stmt_hash_scratch_bytes(uint32_t K, uint32_t R, uint32_t b);
void step1_stmt_hash(const void* C_ser, const void* rows_ser, uint32_t k0, uint32_t K, uint32_t R, uint32_t b,
                     void* scratch, void* hstmt, cudaStream_t s);
void step1_block_r(const void* hstmt, uint32_t k0, uint32_t K, uint32_t R, uint32_t b, void* bvec, cudaStream_t s);
// one thread per step1_miller_group(h) pairs of a product (multi-pair Miller loop); the outputs are
// the products over those groups, in pair order
uint32_t step1_miller_group(uint64_t n, uint32_t h, const EngineLimits& lim);
void step1_miller(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h, uint32_t group, void* out_fq12,
                  cudaStream_t s);
// the same Miller loops with one warp per pair (few pairs: latency)
void round_miller_w(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h, void* out_fq12, cudaStream_t s);
// L_j.1 / R_j.1 terms at the support of the b vectors of blocks k0 .. k0 + K - 1 (blocks of size b),
// dense per-block layout
void step1_sparse_terms(const void* A, const void* bvec, uint32_t k0, uint32_t K, uint32_t R, uint32_t h, uint32_t b,
                        void* out_g1j, cudaStream_t s);
// round j's Miller values (returns how many: K 2h, or fewer when pairs were grouped)
uint64_t step1_miller_g(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h, void* ml_out,
                        cudaStream_t s);
void step1_g1_out(const void* sp_g1j, uint32_t K, int j, void* blocks, size_t bopen_len, cudaStream_t s);
void step1_gt_out(const void* ml_fq12, uint32_t K, int j, void* blocks, size_t bopen_len, cudaStream_t s);
// Round j's folds.  For rounds of at most FOLD_COMB_MAX points, step1_fold_pre forms the comb tables
// of the round's bases in `comb` (fold_comb_bytes(n_max) bytes for up to n_max points) beside the
// round's pairings, and step1_fold then adds one table entry per window; other rounds run the
// whole scalar multiplications after the challenge.
constexpr uint32_t FOLD_COMB_MAX = 256;
size_t fold_comb_bytes(uint32_t n_max);
void step1_fold_pre(const void* A, const void* v, void* comb, uint32_t n_max, uint32_t K, uint32_t R, uint32_t h,
                    cudaStream_t s);
void step1_fold(void* A, void* v, void* bvec, const void* x_mont, const void* xinv_mont, uint32_t K, uint32_t R,
                uint32_t h, const void* comb, uint32_t n_max, cudaStream_t s);
// Look-ahead rounds (lookahead.cuh): round j's record from round j-1's state (half-length h = 2 h2)
// and challenge.  Before the challenge: la_miller (the 8 K h2 Miller values by class; then pairwise
// products to 8 K and their final exponentiations, fe), la_sparse (the 6 K (4 h2) G1 terms; then
// pairwise sums to 6 K, affine, acc; the caller zeroes out_g1j first), la_pre (the shifted bases of the 4-part GT exponentiations and
// G1 multiplications: gpre 12 K Fq12, acc2 12 K G1).  After it: la_gt (the 16 K exponentiation
// parts, pwp) and la_out (round j's record).
void la_miller(const void* A, const void* v, uint32_t K, uint32_t R, uint32_t h2, void* out_fq12, cudaStream_t s);
void la_sparse(const void* A, const void* bvec, uint32_t k0, uint32_t K, uint32_t R, uint32_t h2, uint32_t b,
               void* out_g1j, cudaStream_t s);
void la_pre(const void* fe_fq12, const void* acc_g1a, uint32_t K, void* gpre_fq12, void* acc2_g1a, cudaStream_t s);
void la_gt(const void* fe_fq12, const void* gpre_fq12, const void* x_mont, const void* xinv_mont, uint32_t K,
           void* pwp_fq12, cudaStream_t s);
void la_out(const void* fe_fq12, const void* pwp_fq12, const void* acc_g1a, const void* acc2_g1a, const void* x_mont,
            const void* xinv_mont, uint32_t K, int j, void* blocks, size_t bopen_len, cudaStream_t s);
void step1_challenge(void* blocks, size_t bopen_len, uint32_t K, int j, void* xprev, void* x_mont, void* xinv_mont,
                     void* xinv_all, int log_r, cudaStream_t s);
void step1_kzg(const void* A, const void* v, const void* xprev, const void* xinv_all, uint32_t K, uint32_t R,
               int log_r, void* blocks, size_t bopen_len, void* pcoef, void* q_canon, cudaStream_t s);
void step1_w_terms(const void* g2pow, const void* q_canon, uint32_t K, uint32_t R, void* out_g2j, cudaStream_t s);
// the same terms from the comb tables of g2pow (g2_comb_tables): one table entry per position
void step1_w_comb(const void* tab, const void* q_canon, uint32_t K, uint32_t R, void* out_g2j, cudaStream_t s);
// comb tables of n fixed G2 points (64 positions x 16 entries each, g2_comb_bytes(n) bytes), through
// a scratch of n 64 projective points
constexpr uint32_t G2_COMB_MAX_R = 1024;        // setups with R <= this keep the W proofs' comb tables
size_t g2_comb_bytes(uint32_t n);
size_t g2_comb_chain_bytes(uint32_t n);
void g2_comb_tables(const void* pts_g2a, uint32_t n, void* chain_scratch, void* tab, cudaStream_t s);
// Commit by fixed-base combs of the bases Lambda_a (k_lamcomb.cu): lam_comb_tables builds, at setup,
// 32 windows x 256 affine entries per base (lam_comb_bytes(M); scratch lam_comb_scratch_bytes(M));
// lam_comb_partials writes lam_comb_parts() Jacobian partial sums per (row j, base a) at
// partial[(j M + a) parts + q], whose sum over (a, q) is C_j
constexpr uint32_t LAM_COMB_MAX_M = 1024;       // setups with M <= this keep the commit's comb tables
size_t lam_comb_bytes(uint32_t M);
size_t lam_comb_scratch_bytes(uint32_t M);
void lam_comb_tables(const void* bases_g1a, uint32_t M, void* scratch, void* tab, cudaStream_t s);
void lam_comb_partials(const void* tab, const void* m_canon, uint32_t R, uint32_t M, void* partial_g1j, cudaStream_t s);
uint32_t lam_comb_parts();

// ---- Step 2
void step2_leaves(const void* m_canon, uint32_t R, uint32_t M, void* row_tree, cudaStream_t s);
void tree_level(void* trees, uint32_t ntrees, uint32_t leaves, int level, cudaStream_t s);
void step2_row_leaves(const void* row_tree, const void* rows_ser, uint32_t R, uint32_t M, void* top_tree,
                      cudaStream_t s);
void step2_rj(const void* top_tree, uint32_t R, void* rj, cudaStream_t s);
void step2_randomize(const void* m_mont, const void* rj, uint32_t R, uint32_t M, void* g, cudaStream_t s);
void step2_d0(const void* rows_g1a, const void* rj, uint32_t R, void* D_g1a, cudaStream_t s);
void step2_fold_g(void* g, uint32_t R, uint32_t M, int h, cudaStream_t s);
void step2_fold_d(void* D_g1a, uint32_t R, int h, cudaStream_t s);
void step2_pst_terms(const void* g, const void* lam, uint32_t R, uint32_t M, int log_c, void* out_g1j,
                     cudaStream_t s);
void step2_gstar_ser(const void* g, uint32_t R, uint32_t M, void* out, cudaStream_t s);

// ---- assembly: proofs i0..i0+count-1 back to back
struct ProofLayout {
    uint32_t R, M, b, K;
    int log_n, log_r, log_c;
    size_t bopen_len;
};
void assemble(const ProofLayout& L, const void* rows_ser, const void* blocks, const void* row_tree,
              const void* top_tree, const void* D_ser, const void* g, const void* pst_ser, uint64_t i0, uint64_t count,
              void* out, cudaStream_t s);
size_t proof_len(const ProofLayout& L, uint64_t i);


// ---- multi-scalar multiplication (batched Pippenger; shape in msm.h).  G1: parts = 2, part_bits
// = 129, fmul = 1; G2: parts = 4, part_bits = 65, fmul = 3.
MsmShape msm_shape(uint64_t n, uint32_t nbatch, uint64_t npts, int c, int parts = 2, int part_bits = 129);
size_t msm_scratch_bytes(const MsmShape& sh);
size_t msm_scratch_bytes_g2(const MsmShape& sh);
int msm_window_model(uint64_t n, uint32_t nbatch, int parts = 2, int part_bits = 129, double fmul = 1.0);
// bases: 2 npts affine G1 [P_i | -phi(P_i)]; k_canon: n nbatch x 8 u32; out_g1a / ser_out optional
void msm_g1(const void* bases, const void* k_canon, const MsmShape& sh, void* scratch, void* out_g1a, void* ser_out,
            cudaStream_t s);
// bases: 4 npts affine G2 [(-1)^h psi^h(Q_i)]; serialised result j at ser_out + j ser_stride
void msm_g2(const void* bases, const void* k_canon, const MsmShape& sh, void* scratch, void* out_g2a, void* ser_out,
            size_t ser_stride, cudaStream_t s);
// bases table from n serialised points (err |= 1 on a bad point); or the second half from the first
void msm_bases_load(const void* be96, uint64_t n, void* tab, uint32_t* err, cudaStream_t s);
void msm_bases_endo(void* tab, uint64_t n, cudaStream_t s);
// G2 bases table (4 n points) from nvalid <= n affine points, the rest identity
void msm_bases_g2(const void* pts, uint64_t nvalid, uint64_t n, void* tab, cudaStream_t s);

// ---- evaluation proof at a point (eval.cu)
void eval_point(const void* r_be, int log_n, void* r_mont, uint32_t* err, cudaStream_t s);
void eval_weights(const void* r_mont, int log_r, int log_c, void* T_mont, void* T_canon, cudaStream_t s);
void eval_ftable(const void* m_mont, const void* T_mont, uint32_t R, uint32_t M, void* F, cudaStream_t s);
void eval_bvec(const void* C_ser, const void* r_be, int log_n, const void* CF_ser, const void* T_mont, uint32_t R,
               void* r0, void* bvec, cudaStream_t s);
void eval_pst_fold(void* F, const void* r_mont, int log_c, void* q, void* y_out, cudaStream_t s);
void eval_pst_terms(const void* q, const void* lam, uint32_t M, void* out, cudaStream_t s);

// ---- VC.Verify (verify.cu).  One proof: result word 0 = 0 if accepted.
size_t verify_scratch_bytes(uint32_t b, int lr, int lc);
void verify_one(const void* proof, const void* C_be, const void* mi_be, uint32_t nk, int lr, int lc, uint32_t b,
                uint64_t i, uint32_t M, uint32_t k, uint32_t lo, const void* g1beta, const void* g2tau, void* scratch,
                uint32_t* result, cudaStream_t s);
// FC.BVerify of one block: blk = its nk row commitments, fc = pi_{C_k}; result word 0 = 0 if accepted
size_t verify_block_scratch_bytes(uint32_t b, int lr);
void verify_block(const void* blk, const void* fc, const void* C_be, uint32_t nk, int lr, uint32_t b, uint32_t k,
                  uint32_t lo, const void* g1beta, void* scratch, uint32_t* result, cudaStream_t s);
// The evaluation proof at r (proof = y | C_F | pi_FC | pi_PST, r log_n x 32 B big-endian); result
// word 0 = 0 if accepted
size_t verify_eval_scratch_bytes(uint32_t R, int lr, int lc, int log_n);
void verify_eval(const void* proof, const void* C_be, const void* r_be, int log_n, int lr, int lc, uint32_t R,
                 const void* g1beta, const void* g2tau, void* scratch, uint32_t* result, cudaStream_t s);
// All N proofs of an OpenAll output (its shared pieces as stored by vc_prove_all) against the
// claimed values m (device, N x 4 little-endian u64): ok_out (host, N bytes, may be null) gets 1
// per accepted proof; returns the number accepted.  each = 1: no PST check is shared.  Synchronises.
size_t verify_all_scratch_bytes(const ProofLayout& L);
uint64_t verify_all(const ProofLayout& L, const void* C_be, const void* m, const void* rows_ser, const void* blocks,
                    const void* row_tree, const void* top_tree, const void* D_ser, const void* g, const void* pst_ser,
                    const void* g1beta, const void* g2tau, int each, void* scratch, void* ok_out, cudaStream_t s);

}  // namespace fpk
