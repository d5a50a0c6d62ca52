// Step 2 of OpenAll (Protocol 1 Step 2 and the Sub-protocol, made non-interactive by the Merkle
// tree of Sec. 4.2) and the assembly of individual proofs.
// Stored trees keep every level: leaves first, then each parent level (offset 2L - 2L/2^l).
#include "k_common.cuh"

namespace fpk {

// element leaf: SHA256("FP-leaf" || u64be(i) || m_i)
__global__ void k_leaves(const fr* m_canon, uint32_t R, uint32_t M, uint8_t* row_tree) {
    uint64_t i = gtid();
    if (i >= (uint64_t)R * M) return;
    uint64_t j = i / M, a = i % M;
    uint8_t buf[7 + 8 + 32];
    const char* tag = "FP-leaf";
    for (int q = 0; q < 7; q++) buf[q] = (uint8_t)tag[q];
    put_be64(buf + 7, i);
    const fr c = m_canon[i];
    for (int w = 0; w < 8; w++) put_be32(buf + 15 + 4 * w, c.v[7 - w]);
    sha256(row_tree + (j * (2 * (uint64_t)M - 1) + a) * 32, buf, sizeof buf);
}

// level l of `ntrees` stored trees of `leaves` leaves each: node = SHA256("FP-node" || left || right)
__global__ void k_tree_level(uint8_t* trees, uint32_t ntrees, uint32_t leaves, int level) {
    uint64_t t = gtid();
    uint32_t width = leaves >> level;
    if (t >= (uint64_t)ntrees * width) return;
    uint64_t tr = t / width, s = t % width;
    uint8_t* base = trees + tr * (2 * (uint64_t)leaves - 1) * 32;
    const uint8_t* ch = base + (tree_off(leaves, level - 1) + 2 * s) * 32;
    uint8_t buf[7 + 64];
    const char* tag = "FP-node";
    for (int q = 0; q < 7; q++) buf[q] = (uint8_t)tag[q];
    for (int q = 0; q < 64; q++) buf[7 + q] = ch[q];
    sha256(base + (tree_off(leaves, level) + s) * 32, buf, sizeof buf);
}

// row leaf: SHA256("FP-row" || s_j || C_j)
__global__ void k_row_leaves(const uint8_t* row_tree, const uint8_t* rows_ser, uint32_t R, uint32_t M,
                             uint8_t* top_tree) {
    uint64_t j = gtid();
    if (j >= R) return;
    const uint8_t* sj = row_tree + (j * (2 * (uint64_t)M - 1) + 2 * (uint64_t)M - 2) * 32;
    uint8_t buf[6 + 32 + 96];
    const char* tag = "FP-row";
    for (int q = 0; q < 6; q++) buf[q] = (uint8_t)tag[q];
    for (int q = 0; q < 32; q++) buf[6 + q] = sj[q];
    for (int q = 0; q < 96; q++) buf[38 + q] = rows_ser[j * 96 + q];
    sha256(top_tree + j * 32, buf, sizeof buf);
}

// r_j = HFr("FP-rho", root || u32be(j))
__global__ void k_rj(const uint8_t* top_tree, uint32_t R, fr* rj) {
    uint64_t j = gtid();
    if (j >= R) return;
    uint8_t buf[36];
    const uint8_t* root = top_tree + (2 * (uint64_t)R - 2) * 32;
    for (int q = 0; q < 32; q++) buf[q] = root[q];
    put_be32(buf + 32, (uint32_t)j);
    rj[j] = hash_to_fr("FP-rho", 6, buf, 36, nullptr, 0, nullptr, 0);
}

// g_j = r_j f_j (Eq. ProverRand) -- fold-tree level 0
__global__ void k_randomize(const fr* m_mont, const fr* rj, uint32_t R, uint32_t M, fr* g) {
    uint64_t i = gtid();
    if (i >= (uint64_t)R * M) return;
    g[i] = fr_mul(rj[i / M], m_mont[i]);
}

// D_j = C_j^{r_j} (Eq. ProverRand)
__global__ void __launch_bounds__(64) k_d0(const g1a* rows, const fr* rj, uint32_t R, g1a* D) {
    uint64_t j = gtid();
    if (j >= R) return;
    uint32_t kw[8];
    fr_canon_words(kw, rj[j]);
    D[j] = g1_affine(g1_mul(rows[j], kw));
}

// Sub-protocol: g_w = g_wl + g_wr for every node at level h (all nodes kept)
__global__ void k_fold_g(fr* g, uint32_t R, uint32_t M, int h) {
    uint64_t t = gtid();
    uint32_t width = R >> h;
    if (t >= (uint64_t)width * M) return;
    uint64_t s = t / M, a = t % M;
    uint64_t w = tree_off(R, h) + s, wl = tree_off(R, h - 1) + 2 * s;
    g[w * M + a] = fr_add(g[wl * M + a], g[(wl + 1) * M + a]);
}
// D_w = D_wl D_wr
__global__ void __launch_bounds__(64) k_fold_d(g1a* D, uint32_t R, int h) {
    uint64_t s = gtid();
    if (s >= (R >> h)) return;
    uint64_t w = tree_off(R, h) + s, wl = tree_off(R, h - 1) + 2 * s;
    D[w] = g1_affine(g1_madd(g1_from_affine(D[wl]), D[wl + 1]));
}

// HyperEval on g* (PST at every hypercube point): level t, prefix p < M/2^(t+1), c < 2^t:
// term = (g*[(2p+1) 2^t + c] - g*[2p 2^t + c]) * Lambda_t[c]; flat index t*(M/2) + p*2^t + c.
__global__ void __launch_bounds__(64) k_pst_terms(const fr* g, const g1a* lam, uint32_t R, uint32_t M, int log_c,
                                                  g1j* out) {
    uint64_t idx = gtid();
    uint64_t half = M / 2;
    if (idx >= (uint64_t)log_c * half) return;
    int t = (int)(idx / half);
    uint64_t rem = idx % half, p = rem >> t, c = rem & ((1ull << t) - 1);
    const fr* gs = g + (2 * (uint64_t)R - 2) * M;
    uint64_t w = 1ull << t;
    fr q = fr_sub(gs[(2 * p + 1) * w + c], gs[2 * p * w + c]);
    g1j res;
    if (fr_is_zero(q)) {
        jac_set_inf(res);
    } else {
        uint32_t kw[8];
        fr_canon_words(kw, q);
        res = g1_mul(lam[(1ull << t) - 1 + c], kw);
    }
    out[idx] = res;
}

__global__ void k_gstar_ser(const fr* g, uint32_t R, uint32_t M, uint8_t* out) {
    uint64_t a = gtid();
    if (a >= M) return;
    fr_to_be(out + a * 32, g[(2 * (uint64_t)R - 2) * M + a]);
}

void step2_leaves(const void* m_canon, uint32_t R, uint32_t M, void* row_tree, cudaStream_t s) {
    FP_KERNEL("k_leaves", s, k_leaves<<<grid_for((uint64_t)R * M), TPB, 0, s>>>((const fr*)m_canon, R, M, (uint8_t*)row_tree));
}
void tree_level(void* trees, uint32_t ntrees, uint32_t leaves, int level, cudaStream_t s) {
    uint64_t n = (uint64_t)ntrees * (leaves >> level);
    FP_KERNEL("k_tree_level", s, k_tree_level<<<grid_for(n), TPB, 0, s>>>((uint8_t*)trees, ntrees, leaves, level));
}
void step2_row_leaves(const void* row_tree, const void* rows_ser, uint32_t R, uint32_t M, void* top_tree,
                      cudaStream_t s) {
    FP_KERNEL("k_row_leaves", s, k_row_leaves<<<grid_for(R), TPB, 0, s>>>((const uint8_t*)row_tree, (const uint8_t*)rows_ser, R, M,
                                            (uint8_t*)top_tree));
}
void step2_rj(const void* top_tree, uint32_t R, void* rj, cudaStream_t s) {
    FP_KERNEL("k_rj", s, k_rj<<<grid_for(R), TPB, 0, s>>>((const uint8_t*)top_tree, R, (fr*)rj));
}
void step2_randomize(const void* m_mont, const void* rj, uint32_t R, uint32_t M, void* g, cudaStream_t s) {
    FP_KERNEL("k_randomize", s, k_randomize<<<grid_for((uint64_t)R * M), TPB, 0, s>>>((const fr*)m_mont, (const fr*)rj, R, M, (fr*)g));
}
void step2_d0(const void* rows, const void* rj, uint32_t R, void* D, cudaStream_t s) {
    FP_KERNEL("k_d0", s, k_d0<<<grid_for(R, 64), 64, 0, s>>>((const g1a*)rows, (const fr*)rj, R, (g1a*)D));
}
void step2_fold_g(void* g, uint32_t R, uint32_t M, int h, cudaStream_t s) {
    FP_KERNEL("k_fold_g", s, k_fold_g<<<grid_for((uint64_t)(R >> h) * M), TPB, 0, s>>>((fr*)g, R, M, h));
}
void step2_fold_d(void* D, uint32_t R, int h, cudaStream_t s) {
    FP_KERNEL("k_fold_d", s, k_fold_d<<<grid_for(R >> h, 64), 64, 0, s>>>((g1a*)D, R, h));
}
void step2_pst_terms(const void* g, const void* lam, uint32_t R, uint32_t M, int log_c, void* out, cudaStream_t s) {
    uint64_t n = (uint64_t)log_c * (M / 2);
    FP_KERNEL("k_pst_terms", s, k_pst_terms<<<grid_for(n, 64), 64, 0, s>>>((const fr*)g, (const g1a*)lam, R, M, log_c, (g1j*)out));
}
void step2_gstar_ser(const void* g, uint32_t R, uint32_t M, void* out, cudaStream_t s) {
    FP_KERNEL("k_gstar_ser", s, k_gstar_ser<<<grid_for(M), TPB, 0, s>>>((const fr*)g, R, M, (uint8_t*)out));
}

// ------------------------------------------------------------------------------ assembly
size_t proof_len(const ProofLayout& L, uint64_t i) {
    uint32_t j = (uint32_t)(i / L.M), k = j / L.b;
    uint32_t lo = k * L.b, hi = lo + L.b < L.R ? lo + L.b : L.R;
    return (size_t)(hi - lo) * G1_SER + L.bopen_len + DIGEST * L.log_n + 128 * (size_t)L.log_r + G1_SER * L.log_c;
}

FPG_DEV void copy16(uint8_t* dst, const uint8_t* src, size_t n, int lane) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* d4 = reinterpret_cast<uint4*>(dst);
    for (size_t q = lane; q < n / 16; q += 32) d4[q] = s4[q];
}

// one warp per proof; out offsets are the running sum of proof lengths
__global__ void k_assemble(ProofLayout L, const uint8_t* rows_ser, const uint8_t* blocks, const uint8_t* row_tree,
                           const uint8_t* top_tree, const uint8_t* D_ser, const fr* g, const uint8_t* pst_ser,
                           uint64_t i0, uint64_t count, const uint64_t* offsets, uint8_t* out) {
    uint64_t wid = gtid() / 32;
    int lane = threadIdx.x & 31;
    if (wid >= count) return;
    uint64_t i = i0 + wid;
    uint32_t j = (uint32_t)(i / L.M), a = (uint32_t)(i % L.M), k = j / L.b;
    uint32_t lo = k * L.b, hi = min(lo + L.b, L.R);
    uint8_t* o = out + offsets[wid];
    copy16(o, rows_ser + (size_t)lo * G1_SER, (size_t)(hi - lo) * G1_SER, lane);
    o += (size_t)(hi - lo) * G1_SER;
    copy16(o, blocks + (size_t)k * L.bopen_len, L.bopen_len, lane);
    o += L.bopen_len;
    const uint8_t* rt = row_tree + (size_t)j * (2 * (size_t)L.M - 1) * 32;
    for (int l = 0; l < L.log_c; l++) copy16(o + 32 * l, rt + 32 * (tree_off(L.M, l) + ((a >> l) ^ 1)), 32, lane);
    o += 32 * (size_t)L.log_c;
    for (int l = 0; l < L.log_r; l++)
        copy16(o + 32 * l, top_tree + 32 * (tree_off(L.R, l) + ((j >> l) ^ 1)), 32, lane);
    o += 32 * (size_t)L.log_r;
    for (int h = 0; h < L.log_r; h++) {
        uint64_t w = tree_off(L.R, h) + ((j >> h) ^ 1);
        copy16(o + 128 * h, D_ser + w * G1_SER, G1_SER, lane);
        if (lane == 0) fr_to_be(o + 128 * h + 96, g[w * L.M + a]);
    }
    o += 128 * (size_t)L.log_r;
    for (int idx = 0; idx < L.log_c; idx++) {
        int t = L.log_c - 1 - idx;
        uint64_t off = 0;
        for (int q = 0; q < t; q++) off += L.M >> (q + 1);
        copy16(o + 96 * idx, pst_ser + (off + (a >> (t + 1))) * G1_SER, G1_SER, lane);
    }
}

void assemble(const ProofLayout& L, const void* rows_ser, const void* blocks, const void* row_tree,
              const void* top_tree, const void* D_ser, const void* g, const void* pst_ser, uint64_t i0, uint64_t count,
              void* out, cudaStream_t s) {
    // offsets on the host, copied with the call (count is moderate at every call site)
    uint64_t* h_off = nullptr;
    uint64_t* d_off = nullptr;
    cudaMallocHost(&h_off, count * sizeof(uint64_t));
    uint64_t acc = 0;
    for (uint64_t q = 0; q < count; q++) { h_off[q] = acc; acc += proof_len(L, i0 + q); }
    cudaMallocAsync(&d_off, count * sizeof(uint64_t), s);
    cudaMemcpyAsync(d_off, h_off, count * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
    FP_KERNEL("k_assemble", s, k_assemble<<<grid_for(count * 32, 128), 128, 0, s>>>(L, (const uint8_t*)rows_ser, (const uint8_t*)blocks,
                                                         (const uint8_t*)row_tree, (const uint8_t*)top_tree,
                                                         (const uint8_t*)D_ser, (const fr*)g,
                                                         (const uint8_t*)pst_ser, i0, count, d_off, (uint8_t*)out));
    cudaFreeAsync(d_off, s);
    cudaStreamSynchronize(s);
    cudaFreeHost(h_off);
}

}  // namespace fpk
