// Setup, commit-MSM terms and the generic group kernels (pairwise reductions, normalisation,
// serialisation).
#include "k_common.cuh"
#include "group_ec.cuh"

namespace fpk {

// ------------------------------------------------------------------------------ setup
// SplitMix64 (Steele, Lea, Flood 2014), and Fr draws by rejection of four outputs with the top
// word masked to 63 bits.
__device__ uint64_t splitmix_next(uint64_t& st) {
    uint64_t z = (st += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_trapdoor(uint64_t seed, int log_c, fr* trap) {
    if (gtid() != 0) return;
    uint64_t st = seed ^ 0x5eed5eedull;
    for (int t = 0; t <= log_c; t++) {          // trap[0] = beta, trap[1 + t] = tau_t
        fr c;
        for (;;) {
            for (int w = 0; w < 4; w++) {
                uint64_t z = splitmix_next(st);
                if (w == 3) z &= 0x7fffffffffffffffull;
                c.v[2 * w] = (uint32_t)z;
                c.v[2 * w + 1] = (uint32_t)(z >> 32);
            }
            if (fr_canonical_lt_r(c)) break;
        }
        trap[t] = fr_to_mont(c);
    }
}

// lam_scal[idx] for idx < 2M - 1: level t = floor(log2(idx + 1)), c = idx + 1 - 2^t,
// eq_t(c, tau) = prod_{s<t} (c_s tau_s + (1 - c_s)(1 - tau_s)); pow_scal[i] = beta^i.
__global__ void k_setup_scalars(const fr* trap, int log_r, int log_c, fr* lam_scal, fr* pow_scal, fr* tau_scal,
                                fr* beta_scal) {
    const uint64_t i = gtid();
    const uint64_t M = 1ull << log_c, R = 1ull << log_r;
    fr one; fr_one(one);
    if (i < 2 * M - 1) {
        int t = 63 - __clzll(i + 1);
        uint64_t c = i + 1 - (1ull << t);
        fr acc = one;
        for (int s = 0; s < t; s++) {
            fr tau = trap[1 + s];
            acc = fr_mul(acc, ((c >> s) & 1) ? tau : fr_sub(one, tau));
        }
        lam_scal[i] = fr_from_mont(acc);
    }
    if (i < 2 * R - 1) {
        fr beta = trap[0], acc = one;
        for (int bit = 20; bit >= 0; bit--) {
            acc = fr_mul(acc, acc);
            if ((i >> bit) & 1) acc = fr_mul(acc, beta);
        }
        pow_scal[i] = fr_from_mont(acc);
    }
    if (i < (uint64_t)log_c) tau_scal[i] = fr_from_mont(trap[1 + i]);
    if (i == 0) beta_scal[0] = fr_from_mont(trap[0]);
}

__global__ void k_g1_gen_mul(const fr* scal, uint32_t n, g1a* out) {
    uint64_t i = gtid();
    if (i >= n) return;
    out[i] = g1_affine(g1_mul(g1_generator(), scal[i].v));
}
__global__ void k_g2_gen_mul(const fr* scal, uint32_t n, g2a* out) {
    uint64_t i = gtid();
    if (i >= n) return;
    out[i] = g2_affine(g2_mul(g2_generator(), scal[i].v));
}

void setup_trapdoor(uint64_t seed, int log_c, void* trap, cudaStream_t s) {
    FP_KERNEL("k_trapdoor", s, k_trapdoor<<<1, 32, 0, s>>>(seed, log_c, (fr*)trap));
}
void setup_scalars(const void* trap, int log_r, int log_c, void* lam_scal, void* pow_scal, void* tau_scal,
                   void* beta_scal, cudaStream_t s) {
    uint64_t n = 2ull << (log_c > log_r ? log_c : log_r);
    FP_KERNEL("k_setup_scalars", s, k_setup_scalars<<<grid_for(n), TPB, 0, s>>>((const fr*)trap, log_r, log_c, (fr*)lam_scal, (fr*)pow_scal,
                                                (fr*)tau_scal, (fr*)beta_scal));
}
void g1_gen_mul(const void* scal, uint32_t n, void* out, cudaStream_t s) {
    if (n) FP_KERNEL("k_g1_gen_mul", s, k_g1_gen_mul<<<grid_for(n, 64), 64, 0, s>>>((const fr*)scal, n, (g1a*)out));
}
void g2_gen_mul(const void* scal, uint32_t n, void* out, cudaStream_t s) {
    if (n) FP_KERNEL("k_g2_gen_mul", s, k_g2_gen_mul<<<grid_for(n, 64), 64, 0, s>>>((const fr*)scal, n, (g2a*)out));
}

// ------------------------------------------------------------------------------ reductions
__global__ void k_g1_pair(const g1j* in, g1j* out, uint64_t n) {
    uint64_t i = gtid();
    if (i < n) out[i] = jac_add(in[2 * i], in[2 * i + 1]);
}
__global__ void k_g2_pair(const g2j* in, g2j* out, uint64_t n) {
    uint64_t i = gtid();
    if (i < n) out[i] = jac_add(in[2 * i], in[2 * i + 1]);
}
void g1_pair_reduce(const void* in, void* out, uint64_t n, cudaStream_t s) {
    if (n) FP_KERNEL("k_g1_pair", s, k_g1_pair<<<grid_for(n), TPB, 0, s>>>((const g1j*)in, (g1j*)out, n));
}
void g2_pair_reduce(const void* in, void* out, uint64_t n, cudaStream_t s) {
    if (n) FP_KERNEL("k_g2_pair", s, k_g2_pair<<<grid_for(n, 64), 64, 0, s>>>((const g2j*)in, (g2j*)out, n));
}

// Latency-bound sums of consecutive points, in one launch per factor of 16 or 32: out[g] = the sum of
// in[gs g .. gs g + gs - 1] (gs <= 32 for G1, <= 16 for G2; inputs past n_in count as the identity).
// G1: a 128-thread block per sum, 16 8-lane groups (group_ec.cuh) each adding two inputs, then a tree
// over the groups; G2: a 256-thread block per sum, 8 warps each adding two inputs, then a tree.  Every
// group of a warp runs every addition (one instruction stream); the unneeded ones are discarded.
__global__ void __launch_bounds__(128) k_g1_tree(const g1j* in, g1j* out, uint64_t n_in, uint32_t gs) {
    __shared__ GEcs<fq> e[16];
    __shared__ GPt<fq> part[16];
    const int grp = threadIdx.x >> 3, lane = threadIdx.x & 7;
    const uint64_t i0 = blockIdx.x * (uint64_t)gs + 2 * grp;
    const bool in0 = 2 * grp < (int)gs && i0 < n_in, in1 = 2 * grp + 1 < (int)gs && i0 + 1 < n_in;
    const GPt<fq> a = in0 ? jac_to_proj(in[i0]) : gec_identity<fq>();
    const GPt<fq> b = in1 ? jac_to_proj(in[i0 + 1]) : gec_identity<fq>();
    GPt<fq> acc = gec_add(e[grp], lane, a, b);
    for (int sh = 8; sh >= 1; sh >>= 1) {
        __syncthreads();
        if (lane == 0) part[grp] = acc;
        __syncthreads();
        const GPt<fq> r = gec_add(e[grp], lane, acc, part[grp < sh ? grp + sh : grp]);
        if (grp < sh) acc = r;
    }
    if (grp == 0 && lane == 0) out[blockIdx.x] = proj_to_jac(acc);
}
__global__ void __launch_bounds__(256) k_g2_tree(const g2j* in, g2j* out, uint64_t n_in, uint32_t gs) {
    __shared__ GEcWs e[8];
    __shared__ GPt<fq2> part[8];
    const int w = threadIdx.x >> 5, L = threadIdx.x & 31;
    const uint64_t i0 = blockIdx.x * (uint64_t)gs + 2 * w;
    const bool in0 = 2 * w < (int)gs && i0 < n_in, in1 = 2 * w + 1 < (int)gs && i0 + 1 < n_in;
    const GPt<fq2> a = in0 ? jac_to_proj(in[i0]) : gec_identity<fq2>();
    const GPt<fq2> b = in1 ? jac_to_proj(in[i0 + 1]) : gec_identity<fq2>();
    GPt<fq2> acc = gecw_add(e[w], L, a, b);
    for (int sh = 4; sh >= 1; sh >>= 1) {
        __syncthreads();
        if (L == 0) part[w] = acc;
        __syncthreads();
        if (w < sh) acc = gecw_add(e[w], L, acc, part[w + sh]);
    }
    if (w == 0 && L == 0) out[blockIdx.x] = proj_to_jac(acc);
}
void g1_tree_reduce(const void* in, void* out, uint64_t n_in, uint32_t gs, cudaStream_t s) {
    const uint64_t n_out = (n_in + gs - 1) / gs;
    if (n_out) FP_KERNEL("k_g1_tree", s, k_g1_tree<<<(unsigned)n_out, 128, 0, s>>>((const g1j*)in, (g1j*)out, n_in, gs));
}
void g2_tree_reduce(const void* in, void* out, uint64_t n_in, uint32_t gs, cudaStream_t s) {
    const uint64_t n_out = (n_in + gs - 1) / gs;
    if (n_out) FP_KERNEL("k_g2_tree", s, k_g2_tree<<<(unsigned)n_out, 256, 0, s>>>((const g2j*)in, (g2j*)out, n_in, gs));
}

__global__ void k_g1j_affine(const g1j* in, g1a* out, uint8_t* ser, size_t stride, uint64_t n) {
    uint64_t i = gtid();
    if (i >= n) return;
    g1a a = g1_affine(in[i]);
    if (out) out[i] = a;
    if (ser) g1a_to_be(ser + i * stride, a);
}
__global__ void k_g2j_affine(const g2j* in, g2a* out, uint8_t* ser, size_t stride, uint64_t n) {
    uint64_t i = gtid();
    if (i >= n) return;
    g2a a = g2_affine(in[i]);
    if (out) out[i] = a;
    if (ser) g2a_to_be(ser + i * stride, a);
}
// the same for few points: a quad of four threads per point shares its inversion (jac_to_affine_quad);
// whole quads leave together, the quad's first lane stores
__global__ void k_g1j_affine_q(const g1j* in, g1a* out, uint8_t* ser, size_t stride, uint64_t n) {
    const uint64_t i = gtid() >> 2;
    if (i >= n) return;
    g1a a;
    jac_to_affine_quad(a.x, a.y, in[i]);
    if ((threadIdx.x & 3) == 0) {
        if (out) out[i] = a;
        if (ser) g1a_to_be(ser + i * stride, a);
    }
}
__global__ void k_g2j_affine_q(const g2j* in, g2a* out, uint8_t* ser, size_t stride, uint64_t n) {
    const uint64_t i = gtid() >> 2;
    if (i >= n) return;
    g2a a;
    jac_to_affine_quad(a.x, a.y, in[i]);
    if ((threadIdx.x & 3) == 0) {
        if (out) out[i] = a;
        if (ser) g2a_to_be(ser + i * stride, a);
    }
}
__global__ void k_g1a_ser(const g1a* in, uint8_t* ser, size_t stride, uint64_t n) {
    uint64_t i = gtid();
    if (i < n) g1a_to_be(ser + i * stride, in[i]);
}
__global__ void k_g2a_ser(const g2a* in, uint8_t* ser, size_t stride, uint64_t n) {
    uint64_t i = gtid();
    if (i < n) g2a_to_be(ser + i * stride, in[i]);
}
// up to AFFINE_QUAD_MAX points a quad per point (a shorter inversion on the latency-bound paths), above
// it a thread per point (the quads' repeated division steps would cost throughput)
constexpr uint64_t AFFINE_QUAD_MAX = 4096;
void g1j_to_affine(const void* in, void* out, void* ser, size_t stride, uint64_t n, cudaStream_t s) {
    if (n && n <= AFFINE_QUAD_MAX)
        FP_KERNEL("k_g1j_affine_q", s, k_g1j_affine_q<<<grid_for(4 * n, 64), 64, 0, s>>>((const g1j*)in, (g1a*)out, (uint8_t*)ser, stride, n));
    else if (n)
        FP_KERNEL("k_g1j_affine", s, k_g1j_affine<<<grid_for(n, 64), 64, 0, s>>>((const g1j*)in, (g1a*)out, (uint8_t*)ser, stride, n));
}
void g2j_to_affine(const void* in, void* out, void* ser, size_t stride, uint64_t n, cudaStream_t s) {
    if (n && n <= AFFINE_QUAD_MAX)
        FP_KERNEL("k_g2j_affine_q", s, k_g2j_affine_q<<<grid_for(4 * n, 64), 64, 0, s>>>((const g2j*)in, (g2a*)out, (uint8_t*)ser, stride, n));
    else if (n)
        FP_KERNEL("k_g2j_affine", s, k_g2j_affine<<<grid_for(n, 64), 64, 0, s>>>((const g2j*)in, (g2a*)out, (uint8_t*)ser, stride, n));
}
void g1a_serialize(const void* in, void* ser, size_t stride, uint64_t n, cudaStream_t s) {
    if (n) FP_KERNEL("k_g1a_ser", s, k_g1a_ser<<<grid_for(n), TPB, 0, s>>>((const g1a*)in, (uint8_t*)ser, stride, n));
}
void g2a_serialize(const void* in, void* ser, size_t stride, uint64_t n, cudaStream_t s) {
    if (n) FP_KERNEL("k_g2a_ser", s, k_g2a_ser<<<grid_for(n), TPB, 0, s>>>((const g2a*)in, (uint8_t*)ser, stride, n));
}

__global__ void k_fr_ser(const fr* in, uint64_t n, uint8_t* out) {
    uint64_t i = gtid();
    if (i < n) fr_to_be(out + 32 * i, in[i]);
}
void fr_serialize(const void* in, uint64_t n, void* out, cudaStream_t s) {
    if (n) FP_KERNEL("k_fr_ser", s, k_fr_ser<<<grid_for(n), TPB, 0, s>>>((const fr*)in, n, (uint8_t*)out));
}

// ------------------------------------------------------------------------------ commit
// m arrives as canonical little-endian limbs; values >= r set *err.
__global__ void k_load_vector(const fr* m, uint64_t n, fr* canon, fr* mont, uint32_t* err) {
    uint64_t i = gtid();
    if (i >= n) return;
    fr c = m[i];
    if (!fr_canonical_lt_r(c)) { atomicOr(err, 1u); fr_zero(c); }
    canon[i] = c;
    mont[i] = fr_to_mont(c);
}
void load_vector(const void* m, uint64_t n, void* canon, void* mont, uint32_t* err, cudaStream_t s) {
    FP_KERNEL("k_load_vector", s, k_load_vector<<<grid_for(n), TPB, 0, s>>>((const fr*)m, n, (fr*)canon, (fr*)mont, err));
}
}  // namespace fpk
