/*
 * flexproofs.h -- C ABI of the GB300 (sm_103a) implementation of FlexProofs' all-proofs pass.
 *
 * FlexProofs (Liu, Zhang; arXiv 2601.03031) commits to a vector m of N = 2^n field elements in
 * two layers: each of the R rows (length M) is committed with PST (a multilinear KZG), and the
 * vector of row commitments C = (C_0 .. C_{R-1}) with the paper's functional commitment FC
 * (Sec. 3).  VC.OpenAll (Protocol 1, Sec. 4.2) then produces all N opening proofs in O(N):
 *   Step 1: one FC.BOpen per block S_k = [k b, (k+1) b) of C,
 *   Step 2: Fiat-Shamir Merkle tree, randomised fold tree over the rows, PST HyperEval.
 * Here R = 2^floor(n/2) and M = 2^ceil(n/2) (R = M = sqrt(N) when n is even, Sec. 4.1).
 *
 * Group: BLS12-381 (the paper used BN_SNARK1).  Every byte string crossing this ABI is canonical
 * big-endian: Fr 32 B, G1 96 B (x || y), G2 192 B (x.c0 || x.c1 || y.c0 || y.c1), GT 576 B in the
 * tower order of Fq12 = Fq6[w]/(w^2 - v), Fq6 = Fq2[v]/(v^3 - (1+u)).  The identity of G1/G2 is
 * all zero bytes.  Vectors of Fr cross as N x 4 little-endian uint64 limbs of canonical values.
 *
 * Conventions of every call:
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is enqueued on it; the
 *     calls below that return data to the host synchronise that stream first.
 *   - Handles are owned by the caller and released with the matching *_free (NULL is ignored).
 *     Commitment and proof handles are released stream-ordered (after the work that uses them,
 *     without blocking the host); public parameters and MSM bases synchronise the device.
 *   - Device memory is allocated by the library (stream-ordered) and freed by *_free.
 *   - On any error nothing is written to *out and no partially built handle is returned.
 *   - All computation runs in this library's CUDA kernels on the current device; there is no
 *     CPU fallback.  If no CUDA device is usable, calls fail with FP_EDEVICE.
 */
#ifndef FLEXPROOFS_H
#define FLEXPROOFS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fp_pp fp_pp;           /* public parameters, device resident (VC.Setup, Eq. vcpp) */
typedef struct fp_commit fp_commit;   /* C in GT, aux = row commitments, and the prover's copy of m */
typedef struct fp_proofs fp_proofs;   /* the shared pieces of all N proofs, device resident */
typedef struct fp_g1_bases fp_g1_bases; /* G1 bases of a multi-scalar multiplication, device resident */

typedef enum {
    FP_OK = 0,
    FP_EINVAL = 1,     /* bad size, b out of range, NULL pointer, buffer too small */
    FP_ENOMEM = 2,     /* device or host allocation failed */
    FP_EDEVICE = 3,    /* a CUDA call failed (message via fp_last_error) */
    FP_ETIMEOUT = 4,   /* a bounded device-side wait gave up */
    FP_EVERIFY = 5,    /* a proof did not verify */
    FP_ERANGE = 6      /* an input scalar was >= r */
} fp_status;

/* VC.Setup (Sec. 4.1, Eq. vcpp; FC.Setup of Sec. 3 with the faster-verification extras).
 * Derives the trapdoor (beta, tau_0..tau_{l_c-1}) from SplitMix64 seeded with seed ^ 0x5eed5eed
 * (beta first, then tau_t in order; each an Fr draw by rejection) and builds on the device:
 *   Lambda_t[c] = g1^{prod_{s<t} (c_s tau_s + (1 - c_s)(1 - tau_s))}, t = 0..l_c  (2M - 1 points),
 *   g1^beta, g2^{beta^i} for i < 2R - 1 (v_i = g2^{beta^{2i}} are the even ones), g2^{tau_t}.
 * log_n in [2, 26]; b in [1, R] is only validated here (any b in that range may be used later).
 * The trapdoor never leaves the device and is discarded before returning. */
fp_status vc_setup(uint32_t log_n, uint32_t b, uint64_t seed, void* stream, fp_pp** out);

/* VC.Setup for N = R M split into R = 2^log_r segments of M = 2^log_c elements (OpenAll for
 * sub-arrays, Sec. 4.4, partitions m into any number of equal segments; vc_setup is the split
 * log_r = floor(log_n / 2)).  Same trapdoor stream as vc_setup, so every table is a prefix of the
 * tables of any setup with at least as many rows and columns.  1 <= log_r <= 13, 1 <= log_c,
 * log_r + log_c <= 26; b in [1, R].  Every call that takes an fp_pp works on any split. */
fp_status vc_setup_split(uint32_t log_r, uint32_t log_c, uint32_t b, uint64_t seed, void* stream, fp_pp** out);

/* A view of `pp` for a smaller size 2^log_n (2 <= log_n <= pp's): the same trapdoor, so every table
 * of the smaller setup is a prefix of the larger one's (Lambda_t for t <= l_c, g2^{beta^i} for
 * i < 2R - 1, g2^{tau_t} for t < l_c) and the view shares them; it owns only a small MSM table
 * (2M points).  One resident SRS then serves jobs of every smaller N.  The view must be freed
 * (fp_pp_free) before its parent.  Synchronises the legacy default stream. */
fp_status vc_pp_view(const fp_pp* pp, uint32_t log_n, fp_pp** out);

/* vc_pp_view for any split: log_r <= the parent's log_r and log_c <= the parent's log_c
 * (FP_EINVAL otherwise). */
fp_status vc_pp_view_split(const fp_pp* pp, uint32_t log_r, uint32_t log_c, fp_pp** out);

/* Serialised public parameters (synchronises): Lambda (2M-1) x 96 || g1^beta 96 ||
 * g2^{beta^i} (2R-1) x 192 || g2^{tau_t} l_c x 192.  *len receives the size; out may be NULL to
 * query it. */
fp_status vc_pp_export(const fp_pp* pp, uint8_t* out, size_t cap, size_t* len);
fp_status vc_pp_dims(const fp_pp* pp, uint32_t* log_n, uint32_t* R, uint32_t* M);

/* VC.Commit (Sec. 4.1, Eqs. genCi, genC): C_j = PC.Commit(f_j) = sum_a m[j M + a] Lambda_{l_c}[a]
 * and C = FC.Commit(C) = prod_j e(C_j, g2^{beta^{2j}}).
 * m: N x 4 little-endian uint64 canonical Fr values, on the host (on_device = 0, copied in) or on
 * the current device (on_device = 1, borrowed only for the duration of the enqueued work).
 * The returned handle keeps a device copy of m for OpenAll.  A value >= r gives FP_ERANGE
 * (checked on the device; the call then synchronises). */
fp_status vc_commit(const fp_pp* pp, const uint64_t* m, int on_device, void* stream, fp_commit** out);

/* vc_commit without the synchronisation: the work is only enqueued on `stream`, and the range check
 * of m is reported by vc_commit_status (which waits for this commitment's work only). */
fp_status vc_commit_async(const fp_pp* pp, const uint64_t* m, int on_device, void* stream, fp_commit** out);
fp_status vc_commit_status(const fp_commit* cm);   /* FP_OK, or FP_ERANGE if a value of m was >= r */

/* C (576 B) and, if rows != NULL, the R row commitments (R x 96 B).  Synchronises. */
fp_status vc_commit_get(const fp_commit* cm, uint8_t* gt576, uint8_t* rows);

/* VC.OpenAll (Protocol 1 with the unit-vector shortcut of Sec. 4.3 and the Merkle-tree
 * Fiat-Shamir of Sec. 4.2) for batch size b in [1, R].  Enqueues all work and returns; the shared
 * pieces stay on the device:
 *   - per block k < ceil(R/b): pi_{C_k} = ({L_j, R_j}_{j=1..l_R}, A_l, v_l, W),
 *   - the two-level Merkle tree, the fold tree (g_w, D_w for every node), the PST proofs of g*. */
fp_status vc_prove_all(const fp_pp* pp, const fp_commit* cm, uint32_t b, void* stream, fp_proofs** out);

/* VC.Verify of one proof on the GPU (Sec. 4.2 verification: the Merkle path to the Fiat-Shamir
 * root and r_j, FC.BVerify of block k = (i / M) / b with the b_l shortcut of Sec. 4.3 and the fast
 * verification of v_l (Sec. 3), and PST.Verify of column a = i mod M for D* and y* (Sec. 4.2,
 * Eq. VerifierRand)).
 *   C: 576-byte commitment; m_i: the claimed value, 4 little-endian uint64 (canonical Fr);
 *   proof / len: the bytes of vc_proof_get (host pointers).
 * Returns FP_OK if the proof verifies, FP_EVERIFY if it does not (a check fails, a serialised
 * element is not canonical or not on its curve, m_i >= r, or len is not the proof length for (b, i)),
 * FP_EINVAL for bad arguments.  Synchronises `stream`. */
fp_status vc_verify(const fp_pp* pp, const uint8_t* C, uint32_t b, uint64_t i, const uint64_t m_i[4],
                    const uint8_t* proof, size_t len, void* stream);

/* VC.Verify of all N proofs of a vc_prove_all result at once.  ok[i] (host, N bytes, may be NULL)
 * receives 1 if proof i -- the bytes vc_proof_get(pf, i) would return -- verifies for the claimed
 * value m[i] against C, else 0: the same verdict as vc_verify(pp, C, b, i, m[i], proof i).
 * *n_ok (may be NULL) receives the number accepted.  The verifiers of one block share pi_{C_k}
 * and those of one column share pi*_a (Protocol 1, Steps 1 and 2), so each block's FC.BVerify runs
 * once, and one PST.Verify per column serves every proof whose (root, D*, y*) equal those of the
 * column's row-0 proof; any other proof (say, a wrong claimed value) gets a PST.Verify of its own.
 *   C: 576-byte commitment (host); m: N x 4 little-endian uint64 claimed values, on the host
 *   (on_device = 0) or the current device (on_device = 1); a value >= r fails its proof only.
 *   flags: 0, or 1 = give every proof its own PST.Verify (no column sharing; slower, same verdicts).
 * pf must come from pp (FP_EINVAL otherwise).  Orders itself after pf's work; synchronises `stream`. */
fp_status vc_verify_all(const fp_pp* pp, const uint8_t* C, const uint64_t* m, int on_device, const fp_proofs* pf,
                        int flags, void* stream, uint8_t* ok, uint64_t* n_ok);

/* OpenAll for several independent jobs at once (no counterpart in the paper: serving-side batching).
 * Job j proves jobs[j].cm (any size; commitments made with views of one SRS, or with separate
 * setups) with batch size jobs[j].b.  Every job runs on its own library stream, forked from and
 * joined back to `stream`, so small latency-bound jobs overlap on the device.  use_graph = 1 captures
 * the whole batch (all jobs' launches) into one CUDA graph on `stream` and launches it once; the
 * call then synchronises `stream`.  outs[j] receives job j's handle, identical in content to
 * vc_prove_all(jobs[j].cm, jobs[j].b).  On error no handle is returned. */
typedef struct {
    const fp_commit* cm;
    uint32_t b;
} fp_job;
fp_status vc_prove_all_batch(uint32_t njobs, const fp_job* jobs, int use_graph, void* stream, fp_proofs** outs);
/* Host wall-clock phases of this thread's last vc_prove_all_batch call with use_graph = 1, in ms:
 * enqueueing every job's launches into the capture, instantiating the graph, and launching it
 * until `stream` completes (zeros after a call without a graph).  Any pointer may be NULL. */
fp_status fp_batch_last_times(double* capture_ms, double* instantiate_ms, double* run_ms);

/* One proof pi_i alone (the same bytes as vc_proof_get of vc_prove_all's result): Step 1 for the
 * block of i only (FC.BOpen on S_k, k = (i / M) / b), Step 2 in full (it is O(N) either way), then
 * the proof is assembled.  *len receives the proof length; out may be NULL to query it (no device
 * work).  i >= N or b out of range gives FP_EINVAL.  Synchronises `stream`. */
fp_status vc_prove_one(const fp_pp* pp, const fp_commit* cm, uint32_t b, uint64_t i, void* stream, uint8_t* out,
                       size_t cap, size_t* len);

/* OpenAll for sub-arrays (Sec. 4.4): VC.Commit made the R segment commitments C_j, and Step 1
 * alone proves that C_j is the j-th element of the committed vector for the segments of blocks
 * k0 .. k0 + nblocks - 1 (nblocks = 0: every block from k0 on), b segments per block.  The
 * handle holds those blocks' pi_{C_k}; vc_segment_proof_get reads a segment's proof from it.
 * Element proofs (vc_proof_get, vc_proofs_export, vc_verify_all) are refused on it (FP_EINVAL).
 * Enqueues only, like vc_prove_all. */
fp_status vc_open_segments(const fp_pp* pp, const fp_commit* cm, uint32_t b, uint32_t k0, uint32_t nblocks,
                           void* stream, fp_proofs** out);

/* Byte length of segment j's proof under batch size b: the block's row commitments (C_a)_{a in S_k}
 * (96 B each) || pi_{C_k}, k = j / b.  0 for bad arguments.  No device work. */
size_t vc_segment_proof_len(const fp_pp* pp, uint32_t b, uint32_t j);

/* Segment j's proof (host, synchronises) from a vc_open_segments or vc_prove_all handle; the same
 * bytes are the prefix of every element proof of segment j.  FP_EINVAL if j's block was not
 * opened or cap is too small (out = NULL queries *len). */
fp_status vc_segment_proof_get(const fp_proofs* pf, uint32_t j, uint8_t* out, size_t cap, size_t* len);

/* Verifier V_j of OpenAll for sub-arrays, on the GPU: C_j recomputed from the segment m_j (M x 4
 * little-endian uint64 on the host; the MLE commitment of VC.Commit) must equal the block's entry
 * for j, and FC.BVerify of the block (b_l shortcut, fast verification of v_l) must accept.
 * FP_OK if both hold, FP_EVERIFY if not (also for a value of m_j >= r, a wrong length or a
 * malformed element), FP_EINVAL for bad arguments.  Synchronises `stream`. */
fp_status vc_verify_segment(const fp_pp* pp, const uint8_t* C, uint32_t b, uint32_t j, const uint64_t* m_j,
                            const uint8_t* proof, size_t len, void* stream);

/* Evaluation proof of the committed vector's multilinear extension f_m at a point (Sec. 4.4,
 * "Compatibility with a family of zkSNARKs", Eq. fANDfj), for zkSNARKs that encode their inputs
 * as multilinear polynomials.  r: log_n field elements r_0 .. r_{log N - 1}, 32 bytes big-endian
 * canonical each (host); variable k pairs with bit k of i = j M + a, so r_0 .. r_{l_c - 1} are the
 * column variables r_R and the rest the row variables r_L.  With T_j = eq(j, r_L) and
 * F = sum_j T_j f_j, the proof (host, *len = vc_eval_proof_len bytes; out = NULL queries *len) is
 *   y = f_m(r) (32) || C_F = prod_j C_j^{T_j} (96) || the FC proof of C_F = <C, T> (FC.BOpen with
 *   t = 1: r_0 = HFr("FP-r", SHA256("FP-eval" || C || u32be(log N) || r || C_F) || u32be(0)),
 *   b = r_0 T; the layout of pi_{C_k}) || PST.Eval(F, r_R): pi_{l_c-1} .. pi_0 (96 each).
 * A verifier checks FC.BVerify with C_0 = (C, C_F^{r_0}) and weights r_0 T, and
 * e(C_F - y g1, g2) = prod_t e(pi_t, g2^{tau_t} - r_t g2).  FP_ERANGE if an r_k >= r.
 * Synchronises `stream`. */
size_t vc_eval_proof_len(const fp_pp* pp);
fp_status vc_eval_prove(const fp_pp* pp, const fp_commit* cm, const uint8_t* r, void* stream, uint8_t* out,
                        size_t cap, size_t* len);

/* The verifier of vc_eval_prove's proof on the GPU: FC.BVerify of C_F = <C, T> (b_l shortcut, fast
 * verification of v_l) and PST.Verify of y at r_R.  C: 576-byte commitment, r as for vc_eval_prove,
 * proof / len: host bytes.  FP_OK if both hold, FP_EVERIFY if not (also for a wrong length, an
 * r_k >= r, y >= r or a malformed element), FP_EINVAL for bad arguments.  Synchronises `stream`. */
fp_status vc_eval_verify(const fp_pp* pp, const uint8_t* C, const uint8_t* r, const uint8_t* proof, size_t len,
                         void* stream);

/* Byte length of proof i under batch size b (no device work). */
size_t vc_proof_len(const fp_pp* pp, uint32_t b, uint64_t i);

/* Assemble pi_i (synchronises): block (C_a)_{a in S_k} || pi_{C_k} || Merkle path (l_c row-tree
 * digests then l_R top-tree digests, leaf-up) || l_R sibling pairs (D_w 96 B, g_w[a] 32 B)
 * leaf-up || PST proof (pi_{l_c-1} .. pi_0), with j = i / M, a = i mod M, k = j / b. */
fp_status vc_proof_get(const fp_proofs* pf, uint64_t i, uint8_t* out, size_t cap, size_t* len);

/* Assemble proofs i0 .. i0+count-1 back to back into `out` (host memory, synchronises).  Proof
 * lengths differ only for the last, truncated block; *len receives the total byte count. */
fp_status vc_proofs_export(const fp_proofs* pf, uint64_t i0, uint64_t count, uint8_t* out, size_t cap, size_t* len);

/* Device-to-host copy of the shared proof state (synchronises), the compact result of OpenAll
 * (Protocol 1 Steps 1 and 2 with the Sub-protocol and HyperEval, Sec. 4.2); every element proof is
 * a selection of these bytes.  Layout, all canonical big-endian, concatenated in this order:
 *   K x bopen_len   pi_{C_k} of every block k (zeros for blocks a vc_open_segments call did not open)
 *   R x (2M-1) x 32 the per-row Merkle trees, each leaves first, then every parent level in turn
 *                   (level l of a tree over n leaves at offset 2n - 2n/2^l)
 *   (2R-1) x 32     the tree over the row leaves, same level layout (the root last)
 *   R x 32          r_j
 *   (2R-1) x 96     D_w for every fold-tree node w (same node order: level h node s at 2R - 2R/2^h + s)
 *   (2R-1) x M x 32 g_w for every node, in that node order
 *   (M-1) x 96      HyperEval's PST quotient commitments, level t = 0 .. l_c-1, prefix p at
 *                   sum_{s<t} M/2^(s+1) + p
 * *len receives the size; out may be NULL to query it.  FP_EINVAL for a handle without Step 2. */
fp_status vc_proofs_state(const fp_proofs* pf, uint8_t* out, size_t cap, size_t* len);

/* Pieces for parity checks (synchronise): the Merkle root (32 B), r_j (R x 32 B), g* (M x 32 B)
 * and D* (96 B); any pointer may be NULL. */
fp_status vc_proofs_step2_parts(const fp_proofs* pf, uint8_t* root, uint8_t* rj, uint8_t* gstar, uint8_t* dstar);

/* Allocation-free variant of the row commitments of vc_commit (no counterpart in the paper).
 * For callers that must not allocate device memory: code running where cudaMalloc/cudaFree are
 * unavailable or forbidden -- e.g. a host application whose allocator owns all device memory, or a
 * latency-critical loop that cannot afford the implicit synchronisation an allocation may cause.
 * Computes C_j = sum_a m[j M + a] Lambda_{l_c}[a] for every row j and writes the R rows serialised
 * (R x 96 B, canonical big-endian, identity = zeros) to rows_dev.
 *   m_dev:   device pointer, N x 4 little-endian uint64 canonical Fr values (read only).
 *   rows_dev: device pointer, R x 96 bytes (written).
 * Limit: N = R * M <= 2^14 (larger sizes return FP_EINVAL).  Scratch is one file-scope device array
 * (about 3.5 MB) that every GPU loading the library holds until the process exits.  The first
 * call on a device looks up that array's device address with the device current, so make the first
 * call before any stream capture.  All calls share the array and it keeps the last call's contents
 * (the status word is cleared by each call): calls that overlap on the GPU race -- serialise them.
 * A value >= r gives FP_ERANGE.  Synchronises `stream`.  Allocates no device memory. */
fp_status vc_commit_rows_noalloc(const fp_pp* pp, const uint64_t* m_dev, uint8_t* rows_dev, void* stream);

/* ---- G1 multi-scalar multiplication ----
 * The operation behind PST.Commit (C_j = sum_a m[j M + a] Lambda[a], Sec. 4.1, Eq. genCi) and the
 * PST proofs of HyperEval (Sec. 2), exposed on its own: a batched Pippenger MSM (signed-digit
 * windows over the GLV halves of each scalar, bucket counting sort, bucket accumulation, bucket
 * and window reduction), exact like everything here.
 *
 * fp_g1_bases_from_scalars: bases P_i = s_i g1 for i < n (s: n x 4 little-endian uint64, any
 *   256-bit values; host or device pointer per on_device).  Synchronises.
 * fp_g1_bases_load: bases from n serialised affine points (n x 96 B, canonical big-endian, all-zero
 *   bytes = identity), host or device pointer per on_device.  A coordinate >= p, a point off
 *   y^2 = x^3 + 4 or a point outside the order-r subgroup G1 gives FP_EINVAL (no handle).
 *   Synchronises.
 * Both limit n < 2^30.  The handle holds 2n affine points (P_i and the GLV partner -phi(P_i)),
 * 192 B per base. */
fp_status fp_g1_bases_from_scalars(const uint64_t* s, uint64_t n, int on_device, void* stream, fp_g1_bases** out);
fp_status fp_g1_bases_load(const uint8_t* pts, uint64_t n, int on_device, void* stream, fp_g1_bases** out);
uint64_t fp_g1_bases_count(const fp_g1_bases* P);
void fp_g1_bases_free(fp_g1_bases* P);

/* out[j] = sum_{i<n} k[j n + i] P[(j n + i) mod npts] for j < nbatch, npts = the handle's base count
 * (so nbatch sums over the same n bases when npts = n, or over consecutive slices).
 *   k:   n * nbatch scalars, 4 little-endian uint64 each, any 256-bit values (used mod r).
 *   out: nbatch x 96 B serialised affine points (identity = zeros).
 *   on_device = 1: k and out are device pointers and the call only enqueues (no synchronisation;
 *        scratch is allocated and freed stream-ordered on `stream`).  on_device = 0: both are host
 *        pointers, copied in and out, and the call synchronises.
 *   window: bits per signed digit in [4, 16], or 0 for the library's choice (fp_msm_window).
 * n = 0 gives identities.  Sizes whose bucket lists exceed 2^32 entries give FP_EINVAL. */
fp_status fp_msm_g1(const fp_g1_bases* P, const uint64_t* k, uint64_t n, uint32_t nbatch, int on_device, int window,
                    void* stream, uint8_t* out);
/* The window fp_msm_g1 uses for (n, nbatch) when given 0: the last fp_msm_autotune result for
 * that shape, else a cost model (per-phase throughput and per-thread latency of the field
 * products). */
int fp_msm_window(uint64_t n, uint32_t nbatch);
/* Window of the G2 MSM that forms the v_l proofs W of many blocks (OpenAll Step 1, "Faster
 * verification" of Sec. 3): nbatch sums of n terms, each scalar in four 64-bit GLS parts; the cost
 * model's choice (the launch-name suffix of its kernels is _g2). */
int fp_msm_window_g2(uint64_t n, uint32_t nbatch);
/* Times fp_msm_g1 on `stream` for windows around the model's choice with the given device
 * scalars (n * nbatch), keeps the fastest for (n, nbatch), and returns it (and its time in ms if
 * best_ms != NULL).  Synchronises. */
fp_status fp_msm_autotune(const fp_g1_bases* P, const uint64_t* k_dev, uint64_t n, uint32_t nbatch, void* stream,
                          int* window, double* best_ms);

void fp_pp_free(fp_pp* pp);
void fp_commit_free(fp_commit* cm);
void fp_proofs_free(fp_proofs* pf);

/* Step-1 round schedule of FC.BOpen (Sec. 3, Eq. folding) used by every later call that opens blocks
 * (vc_prove_all, vc_prove_one, vc_prove_all_batch, vc_open_segments, vc_eval_prove); the proofs are
 * byte-identical under every schedule, only the order of the device work differs.
 *   FP_SCHEDULE_DIRECT     (default) round j's pairings after round j-1's fold, one round after
 *                          another.
 *   FP_SCHEDULE_LOOKAHEAD  round j's pairings from round j-1's state before its challenge is known,
 *                          by bilinearity (e(A_L + x A_R, v_L + v_R / x) expanded), so that after
 *                          each challenge only GT exponentiations by x^(+-1) remain on the chain; it
 *                          runs four times a round's Miller loops and final exponentiations beside
 *                          the chain, and on GB300 it is slower than the direct rounds for every
 *                          measured size (kept as an option).
 * A process-wide setting, read when a call enqueues its work.  FP_EINVAL for another value. */
typedef enum { FP_SCHEDULE_DIRECT = 0, FP_SCHEDULE_LOOKAHEAD = 1 } fp_schedule;

/* Engine choice by size (no counterpart in the paper: how the device work is laid out).  Each launch
 * runs its pairings, final exponentiations, fold points or terms either on a latency engine (one
 * 128-thread block or one warp per item: shortest chain, few items) or on a throughput engine (one
 * thread per item: least total work, many items); every engine computes the same values, so these
 * limits change which kernels run and how fast, never the bytes.  Counts are per launch.
 *   miller_block_max / miller_warp_max   Step-1 Miller loops: <= block_max a block each, <= warp_max
 *                                        a warp each, above a thread each (default 1024 / 16383)
 *   miller_group_min                     from this many (and h >= 4), a thread runs 4 pairs of one
 *                                        product with shared squarings (default 2^18)
 *   commit_block_max / commit_warp_max   Commit's R Miller loops, the same way (default 1024 / 16384)
 *   fe_block_max / fe_warp_max           final exponentiations: block / warp / thread (256 / 2^32-1)
 *   pair_block_max                       pairwise Fq12 products: <= a block each, above a thread (2048)
 *   fold_warp_max                        fold points of rounds beyond the split folds (more than 256
 *                                        points): <= a warp (G2) and 8 lanes (G1) each, above a thread
 *                                        (4096)
 *   wterm_warp_max                       terms of the v_l proof W when not by MSM: <= a warp each,
 *                                        above a thread (4096)
 *   msm_chunks                           MSM bucket pass: about this many chunks of the sorted entry
 *                                        list, one thread each (2^17; > 0)
 *   msm_segment_threads                  MSM bucket reduction: at most about this many segment
 *                                        threads (2^15; > 0)
 * A process-wide setting read when a call enqueues its work (set it between calls: a call enqueued
 * concurrently may see either setting).  fp_set_engine_limits(NULL) restores the defaults;
 * FP_EINVAL for a zero msm_chunks or msm_segment_threads. */
typedef struct {
    uint32_t miller_block_max, miller_warp_max, miller_group_min;
    uint32_t commit_block_max, commit_warp_max;
    uint32_t fe_block_max, fe_warp_max;
    uint32_t pair_block_max;
    uint32_t fold_warp_max;
    uint32_t wterm_warp_max;
    uint32_t msm_chunks, msm_segment_threads;
} fp_engine_limits;
fp_status fp_engine_limits_default(fp_engine_limits* out);
fp_status fp_set_engine_limits(const fp_engine_limits* lim);
fp_status fp_get_engine_limits(fp_engine_limits* out);
fp_status fp_set_schedule(int schedule);
int fp_get_schedule(void);

/* ---- diagnostics (no counterpart in the paper: bookkeeping for measurement) ----
 * fp_launch_count: number of CUDA kernel launches this library has made in this process.
 * fp_profile_enable: while on, every launch is bracketed by CUDA events on its stream.
 * fp_profile_report: synchronises those events and writes "name launches total_ms" lines
 * (NUL-terminated, truncated to cap) and returns the size needed; the totals are cleared only
 * by a call that writes them out (out != NULL, cap > 0). */
uint64_t fp_launch_count(void);
void fp_profile_enable(int on);
size_t fp_profile_report(char* out, size_t cap);
/* fp_profile_launches: one "name start_ms ms" line per launch that fp_profile_report has
 * synchronised, in the order the launches were issued, the start measured from the first listed
 * launch's start (NUL-terminated, truncated to cap); returns the size needed and clears the list
 * only by a call that writes it out (out != NULL, cap > 0). */
size_t fp_profile_launches(char* out, size_t cap);
/* Measured rate of the 32-bit integer multiply-add pipe on the current device (lane operations
 * per second, independent chains, all SMs), the denominator of the integer roofline.  Returns a
 * fp_status code. */
int fp_imad_probe(double* ops_per_s, double* ms);

/* Measured latency of one Fq Montgomery product on one lane (a chain of dependent products on the
 * current device, CUDA-event timed), in ns: the unit of the latency bound of the lane-parallel
 * engines, whose every round waits for one product.  Returns a fp_status code. */
int fp_fq_mul_latency(double* ns_per_product);
/* The same for one Fq product computed by the four warps of a 128-thread block together (the block
 * engine's cyclotomic squarings), in ns.  Returns a fp_status code. */
int fp_fq_mul_split_latency(double* ns_per_product);

const char* fp_strerror(fp_status s);
/* Text of the last CUDA error seen by this thread's calls (empty if none). */
const char* fp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
