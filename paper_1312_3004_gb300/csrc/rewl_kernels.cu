// rewl_kernels.cu -- sm_103a kernels of the REWL hot path (arXiv:1312.3004, Sec. 2):
//   init_kernel         initial configuration + entry into the walker's window
//   sweep_kernel        K Wang-Landau steps per walker, binary64 on the walker's
//                       chain (the reference sweep; the production sweep is the
//                       fast sweep of rewl_sweep.cu, which reaches the same states)
//   window_check_kernel visited mask, flatness, merge of ln g, f -> sqrt f
//   exchange_kernel     replica exchange between neighbouring windows (Eq. 1),
//                       then the replicas' round-trip counters
//
// Arithmetic contract (shared with the CPU oracle, written independently):
// spins, energies, histograms and random words are integers; ln g, the
// acceptance exponent and the merge are IEEE binary64 with round-to-nearest and
// no fused multiply-add (the library is compiled with --fmad=false).
#include <cstdint>
#include <cstdio>

#include "rewl_internal.cuh"

namespace rewl {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two round multipliers, crosses the
// high halves with words 1 and 3 and the round key, and the key advances by
// the two Weyl increments.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a0 = c0, a2 = c2;
        c0 = __umulhi(0xCD9E8D57u, a2) ^ c1 ^ k0;
        c2 = __umulhi(0xD2511F53u, a0) ^ c3 ^ k1;
        c1 = 0xCD9E8D57u * a2;
        c3 = 0xD2511F53u * a0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Uniform double in [0, 1) from 27 bits of `hi` and 26 bits of `lo`.
__device__ __forceinline__ double unit53(uint32_t hi, uint32_t lo) {
    const unsigned long long v = ((unsigned long long)(hi >> 5) << 26) | (lo >> 6);
    return __ull2double_rn(v) * 0x1p-53;
}

// ---------------------------------------------------------------------------
// Packed spins: BITS = 8 stores spin s in byte s; BITS = 4 in nibble s & 7 of
// 32-bit word s >> 3.
template <int BITS>
__device__ __forceinline__ int spin_get(const uint32_t *w, int s) {
    if (BITS == 8) return reinterpret_cast<const uint8_t *>(w)[s];
    return (int)((w[s >> 3] >> ((s & 7) << 2)) & 15u);
}
template <int BITS>
__device__ __forceinline__ void spin_set(uint32_t *w, int s, int v) {
    if (BITS == 8) {
        reinterpret_cast<uint8_t *>(w)[s] = (uint8_t)v;
    } else {
        const uint32_t sh = (uint32_t)(s & 7) << 2;
        w[s >> 3] = (w[s >> 3] & ~(15u << sh)) | ((uint32_t)v << sh);
    }
}

// Periodic neighbours of site s = y*L + x (Eq. 2 on an L x L torus).
struct Nbrs { int r, l, d, u; };
__device__ __forceinline__ Nbrs neighbours(int s, int L, int N, uint32_t divL) {
    const int y = (int)__umulhi((uint32_t)s, divL);  // s / L, exact for L <= 1024
    const int x = s - y * L;
    Nbrs n;
    n.r = (x == L - 1) ? s - (L - 1) : s + 1;
    n.l = (x == 0) ? s + (L - 1) : s - 1;
    n.d = (y == L - 1) ? s - (N - L) : s + L;
    n.u = (y == 0) ? s + (N - L) : s - L;
    return n;
}

// Energy change of setting site s from `cur` to `nw`: bonds to neighbours equal
// to cur break, bonds to neighbours equal to nw form.
template <int BITS>
__device__ __forceinline__ int delta_e(const uint32_t *w, const Nbrs &n, int cur, int nw) {
    const int a = spin_get<BITS>(w, n.r), b = spin_get<BITS>(w, n.l);
    const int c = spin_get<BITS>(w, n.d), d = spin_get<BITS>(w, n.u);
    return (int)(a == cur) + (int)(b == cur) + (int)(c == cur) + (int)(d == cur) -
           (int)(a == nw) - (int)(b == nw) - (int)(c == nw) - (int)(d == nw);
}

template <int BITS>
__device__ int recount_energy(const uint32_t *w, const Model &M) {
    int sat = 0;
    for (int s = 0; s < M.N; ++s) {
        const Nbrs n = neighbours(s, M.L, M.N, M.divL);
        const int v = spin_get<BITS>(w, s);
        sat += (v == spin_get<BITS>(w, n.r)) + (v == spin_get<BITS>(w, n.d));
    }
    return -sat;
}

// ---------------------------------------------------------------------------
// Initial state: random spins from the seed, then entry into the window.  A
// walker whose window lies below the drawn energy restarts from a uniform
// ground state (E = -2N); it then climbs with single flips that keep
// E <= E' <= E_hi until E >= E_lo.  Entry moves change neither ln g nor H.
// One thread per walker slot; lattices in global memory (runs once).
template <int BITS>
__global__ void init_kernel(Model M, State S) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M.G) return;
    uint32_t *w = S.spins + (size_t)g * M.wpc;
    for (int s0 = 0; s0 < M.N; s0 += 4) {
        const uint4 r = philox((uint32_t)(s0 >> 2), 0u, (uint32_t)g, DOM_INIT, M.key0, M.key1);
        const uint32_t rv[4] = {r.x, r.y, r.z, r.w};
        for (int j = 0; j < 4 && s0 + j < M.N; ++j) spin_set<BITS>(w, s0 + j, (int)__umulhi(rv[j], (uint32_t)M.q));
    }
    int E = recount_energy<BITS>(w, M);
    const int lo = S.e_lo[g / M.m], hi = lo + M.W;
    if (E > hi) {
        const uint4 r = philox(0u, 0u, (uint32_t)g, DOM_ENTRY, M.key0, M.key1);
        const uint32_t c = __umulhi(r.x, (uint32_t)M.q);
        const uint32_t fill = (BITS == 8) ? c * 0x01010101u : c * 0x11111111u;
        for (int j = 0; j < M.wpc; ++j) w[j] = fill;
        E = -2 * M.N;
    }
    const unsigned long long max_moves = 1000ull * (unsigned long long)M.N + 1000000ull;
    for (unsigned long long n = 1; E < lo; ++n) {
        if (n > max_moves) {
            atomicOr(&S.ctl->error, ERR_ENTRY);
            break;
        }
        const uint4 r = philox((uint32_t)n, (uint32_t)(n >> 32), (uint32_t)g, DOM_ENTRY, M.key0, M.key1);
        const int site = (int)__umulhi(r.x, (uint32_t)M.N);
        const int cur = spin_get<BITS>(w, site);
        const int v = (int)__umulhi(r.y, (uint32_t)(M.q - 1));
        const int nw = v + (v >= cur);
        const int En = E + delta_e<BITS>(w, neighbours(site, M.L, M.N, M.divL), cur, nw);
        if (En >= E && En <= hi) {
            spin_set<BITS>(w, site, nw);
            E = En;
        }
    }
    S.cfg_E[g] = E;
    S.slot_cfg[g] = (uint32_t)g;
    // replica g starts in walker g's window
    const int wg = g / M.m;
    S.rt_end[g] = M.h < 2 ? 0 : (wg == 0 ? 1 : (wg == M.h - 1 ? 2 : 0));
    S.rt_trips[g] = 0u;
    S.t[g] = 0ull;
}

// ---------------------------------------------------------------------------
// The hot loop: K standard WL steps per walker (Sec. 2).  One thread per
// walker; a CTA holds P walkers whose lattices, ln g and H live in shared
// memory for the whole launch and are written back at the end.
//
// Per step, with one Philox block (t, t>>32, g, 0):
//   site = r0*N >> 32; new spin v + (v >= cur), v = r1*(q-1) >> 32;
//   E' = E + dE; outside [E_lo, E_hi] -> reject;
//   else accept iff D >= 0 or u < exp(D), D = ln g(E) - ln g(E'), u from r2, r3;
//   then ln g(E) += ln f, H(E) += 1 at the current E.
template <int BITS>
__global__ void __launch_bounds__(256) sweep_kernel(Model M, State S, int P) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (*(volatile unsigned int *)&S.ctl->all_done) return;
    double *s_lng = reinterpret_cast<double *>(smem);
    uint32_t *s_H = reinterpret_cast<uint32_t *>(s_lng + (size_t)P * M.B);
    uint32_t *s_spin = s_H + (size_t)P * M.B;
    const int g0 = blockIdx.x * P;
    const int PB = P * M.B, PW = P * M.wpc;

    for (int i = threadIdx.x; i < PB; i += blockDim.x) {
        const int p = i / M.B, g = g0 + p;
        if (g < M.G && !S.done[g / M.m]) {
            const size_t src = (size_t)g * M.B + (i - p * M.B);
            s_lng[i] = S.lng[src];
            s_H[i] = S.H[src];
        }
    }
    for (int i = threadIdx.x; i < PW; i += blockDim.x) {
        const int p = i / M.wpc, g = g0 + p;
        if (g < M.G && !S.done[g / M.m]) s_spin[i] = S.spins[(size_t)S.slot_cfg[g] * M.wpc + (i - p * M.wpc)];
    }
    __syncthreads();

    const int p = threadIdx.x, g = g0 + p;
    if (p < P && g < M.G && !S.done[g / M.m]) {
        const int w = g / M.m;
        const int lo = S.e_lo[w], hi = lo + M.W;
        const double lnf = S.lnf[w];
        uint32_t *lat = s_spin + (size_t)p * M.wpc;
        double *lg = s_lng + (size_t)p * M.B;
        uint32_t *hg = s_H + (size_t)p * M.B;
        const uint32_t c = S.slot_cfg[g];
        int E = S.cfg_E[c];
        unsigned long long t = S.t[g];
        unsigned long long n_acc = 0;
        unsigned int bad = 0;  // failed bounds checks (debug build)
        const uint32_t N = (uint32_t)M.N, qm1 = (uint32_t)(M.q - 1);
        for (long long k = 0; k < M.K; ++k, ++t) {
            const uint4 r = philox((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)g, DOM_WL, M.key0, M.key1);
            const int site = (int)__umulhi(r.x, N);
            const int cur = spin_get<BITS>(lat, site);
            const int v = (int)__umulhi(r.y, qm1);
            const int nw = v + (v >= cur);
            const int En = E + delta_e<BITS>(lat, neighbours(site, M.L, M.N, M.divL), cur, nw);
            if (En >= lo && En <= hi) {
                const double d = __dsub_rn(lg[REWL_IDX(E - lo, 0, M.B, bad)], lg[REWL_IDX(En - lo, 0, M.B, bad)]);
                bool acc = d >= 0.0;
                if (!acc) {
                    const double u = unit53(r.z, r.w);
                    const double e = exp(d);
                    acc = u < e;
                    if (fabs(u - e) < 1e-14) record_tie(S.ctl, S.tlog, TIE_WL, (unsigned int)g, t);
                }
                if (acc) {
                    spin_set<BITS>(lat, site, nw);
                    E = En;
                    ++n_acc;
                }
            }
            const int b = REWL_IDX(E - lo, 0, M.B, bad);
            lg[b] = __dadd_rn(lg[b], lnf);
            hg[b] += 1u;
        }
        S.cfg_E[c] = E;
        S.t[g] = t;
        atomicAdd(&S.ctl->flips, (unsigned long long)M.K);
        atomicAdd(&S.ctl->accepted, n_acc);
        if (bad) atomicOr(&S.ctl->error, ERR_BOUNDS);
    }
    __syncthreads();

    for (int i = threadIdx.x; i < PB; i += blockDim.x) {
        const int pp = i / M.B, gg = g0 + pp;
        if (gg < M.G && !S.done[gg / M.m]) {
            const size_t dst = (size_t)gg * M.B + (i - pp * M.B);
            S.lng[dst] = s_lng[i];
            S.H[dst] = s_H[i];
        }
    }
    for (int i = threadIdx.x; i < PW; i += blockDim.x) {
        const int pp = i / M.wpc, gg = g0 + pp;
        if (gg < M.G && !S.done[gg / M.m]) S.spins[(size_t)S.slot_cfg[gg] * M.wpc + (i - pp * M.wpc)] = s_spin[i];
    }
}

// ---------------------------------------------------------------------------
// Fixed-weight production (Sec. 3.2: once g(E) is known, configurations are
// sampled with the fixed weights 1/g(E) and distributions H(E, O) recorded).
// Each walker keeps its own final ln g and ln f = 0, so a WL step is a
// Metropolis step inside the window with the same decision as the sweep
// (accept iff D >= 0 or u < exp(D), exp evaluated only when a single-precision
// bracket of -ln u cannot decide); after every step the window's H(E, O)
// counts the current energy and the class of the majority count
// O = max_v #{i : s_i = v} of the configuration, one of n_obins equal integer
// classes of [ceil(N/q), N].  Every window runs, finished or not; H stays 0.
// One thread per walker; lattice, ln g and the spin counts of the walker's
// configuration buffer in global memory (the thread owns that buffer for the
// launch); runs of equal (E, O) are added to H(E, O) with one atomic each.
template <int BITS>
__global__ void __launch_bounds__(256) production_kernel(Model M, State S, int per) {
    // per walkers per CTA (the CTA is a whole number of warps, the rest idle):
    // spread over every SM, since each walker's chain, not a pipe, sets its rate
    const int g = blockIdx.x * per + (int)threadIdx.x;
    if ((int)threadIdx.x >= per || g >= M.G) return;
    const int w = g / M.m;
    const int lo = S.e_lo[w], hi = lo + M.W;
    const uint32_t c = S.slot_cfg[g];
    uint32_t *lat = S.spins + (size_t)c * M.wpc;
    int32_t *cnt = S.cnt + (size_t)c * M.q;
    const double *lg = S.lng + (size_t)g * M.B;
    unsigned long long *heo = S.heo + (size_t)w * M.B * M.n_obins;
    int E = S.cfg_E[c];
    unsigned long long t = S.t[g];
    const int qlo = (M.N + M.q - 1) / M.q;  // ceil(N / q), the smallest majority
    const long long span = (long long)(M.N - qlo + 1);
    int nmax = 0;
    for (int v = 0; v < M.q; ++v) nmax = max(nmax, cnt[v]);
    int key = -1;                     // (bin, class) of the current run of steps
    unsigned long long run = 0, n_acc = 0;
    unsigned int bad = 0;  // failed bounds checks (debug build)
    const uint32_t N = (uint32_t)M.N, qm1 = (uint32_t)(M.q - 1);
    for (long long k = 0; k < M.K; ++k, ++t) {
        const uint4 r = philox((uint32_t)t, (uint32_t)(t >> 32), (uint32_t)g, DOM_WL, M.key0, M.key1);
        const int site = (int)__umulhi(r.x, N);
        const int cur = spin_get<BITS>(lat, site);
        const int v = (int)__umulhi(r.y, qm1);
        const int nw = v + (v >= cur);
        const int En = E + delta_e<BITS>(lat, neighbours(site, M.L, M.N, M.divL), cur, nw);
        if (En >= lo && En <= hi) {
            const double d = __dsub_rn(lg[REWL_IDX(E - lo, 0, M.B, bad)], lg[REWL_IDX(En - lo, 0, M.B, bad)]);
            bool acc = d >= 0.0;
            if (!acc) {
                // The reference decision u < exp(d), taken first against a
                // bracket of -ln u from single precision: uf is u to 2^-23
                // relative (the 24 + 24 bits below carry one rounding, and the
                // dropped 5 bits are under 2^-24 of u once the top 24 bits are
                // not all zero), logf is within one ulp, so |Lf + ln u| is below
                // (Lf + 1) 2^-22.9; the margin (Lf + 1) 2^-18 leaves a factor
                // over 20 for that and for exp's own rounding (one ulp of a
                // double).  Outside the bracket the binary64 comparison can only
                // come out as the bracket says; inside it (about 1e-5 of the
                // decisions) exp(d) decides, as in the reference.
                const unsigned long long U = ((unsigned long long)(r.z >> 5) << 26) | (r.w >> 6);
                const uint32_t top = (uint32_t)(U >> 29);
                int sure = 0;  // 1: accept, -1: reject, 0: take the exact path
                if (top != 0u) {
                    const float uf = fmaf((float)top, 0x1p-24f, (float)((uint32_t)(U >> 5) & 0xffffffu) * 0x1p-48f);
                    const float Lf = -logf(uf);
                    const float margin = (Lf + 1.0f) * 0x1p-18f;
                    const double nd = -d;
                    if (nd < (double)(Lf - margin)) sure = 1;
                    else if (nd >= (double)(Lf + margin)) sure = -1;
                }
                if (sure != 0) {
                    acc = sure > 0;
                } else {
                    const double u = unit53(r.z, r.w);
                    const double e = exp(d);
                    acc = u < e;
                    if (fabs(u - e) < 1e-14) record_tie(S.ctl, S.tlog, TIE_WL, (unsigned int)g, t);
                }
            }
            if (acc) {
                spin_set<BITS>(lat, site, nw);
                E = En;
                ++n_acc;
                const int oc = cnt[cur], nc = cnt[nw] + 1;
                cnt[cur] = oc - 1;
                cnt[nw] = nc;
                if (nc > nmax) {
                    nmax = nc;
                } else if (oc == nmax) {  // the old majority value lost a spin
                    nmax = 0;
                    for (int u = 0; u < M.q; ++u) nmax = max(nmax, cnt[u]);
                }
            }
        }
        const int kk = REWL_IDX(E - lo, 0, M.B, bad) * M.n_obins + (int)((long long)(nmax - qlo) * M.n_obins / span);
        if (kk == key) {
            ++run;
        } else {
            if (run) atomicAdd(&heo[key], run);
            key = kk;
            run = 1;
        }
    }
    if (run) atomicAdd(&heo[key], run);
    S.cfg_E[c] = E;
    S.t[g] = t;
    atomicAdd(&S.ctl->flips, (unsigned long long)M.K);
    atomicAdd(&S.ctl->accepted, n_acc);
    if (bad) atomicOr(&S.ctl->error, ERR_BOUNDS);
}

// Spins of each value in configuration buffer blockIdx.x (production set-up).
template <int BITS>
__global__ void count_spins_kernel(Model M, State S) {
    __shared__ int n[256];
    const int c = blockIdx.x;
    for (int v = threadIdx.x; v < 256; v += blockDim.x) n[v] = 0;
    __syncthreads();
    const uint32_t *lat = S.spins + (size_t)c * M.wpc;
    for (int s = threadIdx.x; s < M.N; s += blockDim.x) atomicAdd(&n[spin_get<BITS>(lat, s)], 1);
    __syncthreads();
    for (int v = threadIdx.x; v < M.q; v += blockDim.x) S.cnt[(size_t)c * M.q + v] = n[v];
}

// ---------------------------------------------------------------------------
// Barrier part 1, one CTA per window (Sec. 2): (a) bins any walker visited
// join the window's mask; (b) walker k is flat iff min H >= p * mean H over the
// mask; (c) when all m walkers are flat: ln g of every bin becomes the mean of
// the m walkers' values (pairwise tree in walker order: stride 1, 2, 4, ...,
// an element without partner passes through; then / m), H <- 0,
// ln f <- ln f / 2 (f -> sqrt f); the window is finished once ln f < ln f_final.
// Under the 1/t rule (SCHED_INV_T, Belardinelli & Pereyra) the criterion of (b)
// is "every mask bin visited" (min H >= 1); at the end of an iteration ln f is
// halved unless the half falls below 1/t, t = WL steps per walker / bins in
// the mask, after which the window follows ln f = 1/t: merge and H <- 0 at
// every barrier, ln f = 1/t with the current t.
constexpr int MAX_M = 256;  // walkers per window (exchange permutation buffer)
constexpr int CHECK_THREADS = 256;

__device__ void window_check_block(const Model &M, const State &S, int w) {
    if (*(volatile unsigned int *)&S.ctl->all_done) return;
    if (S.done[w]) return;
    const int B = M.B, m = M.m, tid = threadIdx.x;
    const size_t base = (size_t)w * m * B;
    uint8_t *mask = S.mask + (size_t)w * B;

    int ovf = 0;
    for (int b = tid; b < B; b += blockDim.x) {
        int vis = 0;
        for (int k = 0; k < m; ++k) {
            const uint32_t hv = S.H[base + (size_t)k * B + b];
            vis |= hv > 0u;
            ovf |= hv >= 0x80000000u;
        }
        if (vis) mask[b] = 1;
    }
    if (__syncthreads_or(ovf)) {
        if (tid == 0) atomicOr(&S.ctl->error, ERR_OVERFLOW);
        return;
    }

    const bool inv_t = M.schedule == SCHED_INV_T;
    const bool follows_1t = inv_t && S.phase[w];
    __shared__ unsigned int r_n[CHECK_THREADS / 32], r_mn[CHECK_THREADS / 32];
    __shared__ unsigned long long r_sum[CHECK_THREADS / 32];
    __shared__ int all_flat;
    __shared__ unsigned int n_bins;  // bins in the window's mask
    if (tid == 0) all_flat = 1;
    for (int k = 0; k < m; ++k) {
        unsigned int n = 0, mn = 0xffffffffu;
        unsigned long long sum = 0;
        const uint32_t *hk = S.H + base + (size_t)k * B;
        for (int b = tid; b < B; b += blockDim.x) {
            if (!mask[b]) continue;
            const uint32_t hv = hk[b];
            n += 1u;
            sum += hv;
            mn = min(mn, hv);
        }
        for (int o = 16; o > 0; o >>= 1) {
            n += __shfl_xor_sync(0xffffffffu, n, o);
            sum += __shfl_xor_sync(0xffffffffu, sum, o);
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        }
        __syncthreads();
        if ((tid & 31) == 0) {
            r_n[tid >> 5] = n;
            r_sum[tid >> 5] = sum;
            r_mn[tid >> 5] = mn;
        }
        __syncthreads();
        if (tid == 0) {
            unsigned int tn = 0, tmn = 0xffffffffu;
            unsigned long long ts = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
                tn += r_n[i];
                ts += r_sum[i];
                tmn = min(tmn, r_mn[i]);
            }
            const bool flat = tn > 0 && (inv_t ? tmn >= 1u : (double)tmn >= M.flatness * ((double)ts / (double)tn));
            if (!flat) all_flat = 0;
            n_bins = tn;
        }
    }
    __syncthreads();
    if (!all_flat && !follows_1t) return;

    // Merge: the pairwise tree is formed in place in the walkers' own rows (they
    // are overwritten by the mean afterwards); each thread owns whole bins.
    for (int b = tid; b < B; b += blockDim.x) {
        double *col = S.lng + base + b;
        for (int stride = 1; stride < m; stride *= 2)
            for (int k = 0; k + stride < m; k += 2 * stride)
                col[(size_t)k * B] = __dadd_rn(col[(size_t)k * B], col[(size_t)(k + stride) * B]);
        const double mean = __ddiv_rn(col[0], (double)m);
        for (int k = 0; k < m; ++k) {
            col[(size_t)k * B] = mean;
            S.H[base + (size_t)k * B + b] = 0u;
        }
    }
    if (tid == 0) {
        double nl;
        if (!inv_t) {
            nl = S.lnf[w] * 0.5;
            S.iter[w] += 1;
        } else {
            const unsigned long long steps = S.t[(size_t)w * m];
            const double one_over_t = steps ? __ddiv_rn((double)n_bins, (double)steps) : 0.0;
            if (follows_1t) {
                nl = one_over_t;
            } else {
                nl = S.lnf[w] * 0.5;
                S.iter[w] += 1;
                if (nl < one_over_t) {
                    S.phase[w] = 1;
                    nl = one_over_t;
                }
            }
        }
        S.lnf[w] = nl;
        if (nl < M.lnf_final) S.done[w] = 1;
    }
}

__global__ void __launch_bounds__(CHECK_THREADS) window_check_kernel(Model M, State S) {
    window_check_block(M, S, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Barrier part 2, one CTA (Sec. 2, Eq. 1): for every window pair (a, a+1)
// with a = round mod 2 and neither window finished, walker k of window a is
// matched with walker pi(k) of window a+1 (pi: Fisher-Yates shuffle, word n of
// the round's draws picks j = word * (i+1) >> 32 for i = m-1 .. 1); if each
// configuration's energy lies in the other walker's window, the pair swaps
// configurations with probability min[1, g_i(E_X) g_j(E_Y) / (g_i(E_Y) g_j(E_X))].
// A swap exchanges the two walkers' buffer ids; ln g and H stay with the walkers.
// Then the round counter advances and the completion flag is refreshed.
constexpr int XCH_THREADS = 1024;

__device__ void exchange_block(const Model &M, const State &S) {
    __shared__ int perm[XCH_THREADS / 32][MAX_M];
    Ctl *ctl = S.ctl;
    if (!M.production && *(volatile unsigned int *)&ctl->all_done) return;
    const unsigned long long round = ctl->round;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int m = M.m, B = M.B;
    unsigned long long tried = 0, acc = 0;
    for (int a = (int)(round & 1ull) + 2 * warp; a + 1 < M.h; a += 2 * nwarps) {
        if (!M.production && (S.done[a] || S.done[a + 1])) continue;  // production: every pair
        int *pi = perm[warp];
        if (lane == 0) {
            for (int k = 0; k < m; ++k) pi[k] = k;
            for (int i = m - 1; i >= 1; --i) {
                const int n = m - 1 - i;
                const uint4 r = philox((uint32_t)round, (uint32_t)(n >> 2), (uint32_t)a, DOM_PERM, M.key0, M.key1);
                const uint32_t word = (n & 3) == 0 ? r.x : (n & 3) == 1 ? r.y : (n & 3) == 2 ? r.z : r.w;
                const int j = (int)__umulhi(word, (uint32_t)(i + 1));
                const int tmp = pi[i];
                pi[i] = pi[j];
                pi[j] = tmp;
            }
        }
        __syncwarp();
        const int lo_a = S.e_lo[a], hi_a = lo_a + M.W;
        const int lo_b = S.e_lo[a + 1], hi_b = lo_b + M.W;
        for (int k = lane; k < m; k += 32) {
            const int gi = a * m + k, gj = (a + 1) * m + pi[k];
            const uint32_t ci = S.slot_cfg[gi], cj = S.slot_cfg[gj];
            const int Ei = S.cfg_E[ci], Ej = S.cfg_E[cj];
            if (!(Ei >= lo_b && Ei <= hi_b && Ej >= lo_a && Ej <= hi_a)) continue;
            const double *li = S.lng + (size_t)gi * B;
            const double *lj = S.lng + (size_t)gj * B;
            const double d = __dadd_rn(__dsub_rn(li[Ei - lo_a], li[Ej - lo_a]), __dsub_rn(lj[Ej - lo_b], lj[Ei - lo_b]));
            const uint4 r = philox((uint32_t)round, (uint32_t)k, (uint32_t)a, DOM_XACC, M.key0, M.key1);
            ++tried;
            bool ok = d >= 0.0;
            if (!ok) {
                const double u = unit53(r.x, r.y), e = exp(d);
                ok = u < e;
                if (fabs(u - e) < 1e-14) record_tie(ctl, S.tlog, TIE_EXCHANGE, (unsigned int)gi, round);
            }
            if (ok) {
                S.slot_cfg[gi] = cj;
                S.slot_cfg[gj] = ci;
                ++acc;
            }
        }
        __syncwarp();
    }
    if (tried) atomicAdd(&ctl->xtried, tried);
    if (acc) atomicAdd(&ctl->xacc, acc);
    __syncthreads();
    // replica round trips: a replica now in the lowest window completes one if
    // it has been in the highest window since it last was in the lowest
    if (M.h >= 2) {
        for (int g = threadIdx.x; g < M.G; g += blockDim.x) {
            const uint32_t c = S.slot_cfg[g];
            const int w = g / m;
            if (w == 0) {
                if (S.rt_end[c] == 2) S.rt_trips[c] += 1u;
                S.rt_end[c] = 1;
            } else if (w == M.h - 1) {
                S.rt_end[c] = 2;
            }
        }
    }
    if (threadIdx.x == 0) {
        ctl->round = round + 1ull;
        unsigned int all = 1u;
        for (int w = 0; w < M.h; ++w) all &= (unsigned int)(S.done[w] != 0);
        ctl->all_done = all;
    }
}

__global__ void __launch_bounds__(XCH_THREADS) exchange_kernel(Model M, State S) { exchange_block(M, S); }

// ---------------------------------------------------------------------------
// Batched forms: many independent instances in one launch.  Every CTA looks up
// its instance in a device table and runs the same block code as above.
__global__ void __launch_bounds__(CHECK_THREADS) batch_check_kernel(const InstDev *inst, const WinItem *wins) {
    const WinItem it = wins[blockIdx.x];
    const Model M = inst[it.inst].M;
    const State S = inst[it.inst].S;
    window_check_block(M, S, it.w);
}

__global__ void __launch_bounds__(XCH_THREADS) batch_exchange_kernel(const InstDev *inst) {
    const Model M = inst[blockIdx.x].M;
    const State S = inst[blockIdx.x].S;
    exchange_block(M, S);
}

// ---------------------------------------------------------------------------
// Unpack / pack walker configurations for state access (walker order).
template <int BITS>
__global__ void get_spins_kernel(Model M, State S, uint8_t *out) {
    const size_t total = (size_t)M.G * M.N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(i / M.N), s = (int)(i - (size_t)g * M.N);
        out[i] = (uint8_t)spin_get<BITS>(S.spins + (size_t)S.slot_cfg[g] * M.wpc, s);
    }
}
template <int BITS>
__global__ void set_spins_kernel(Model M, State S, const uint8_t *in) {
    const size_t total = (size_t)M.G * M.wpc;
    const int per = 32 / BITS;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int g = (int)(i / M.wpc), j = (int)(i - (size_t)g * M.wpc);
        uint32_t word = 0;
        for (int e = 0; e < per; ++e) {
            const int s = j * per + e;
            if (s < M.N) word |= (uint32_t)in[(size_t)g * M.N + s] << (e * BITS);
        }
        S.spins[(size_t)S.slot_cfg[g] * M.wpc + j] = word;
    }
}
template <int BITS>
__global__ void recount_kernel(Model M, State S) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M.G) return;
    const uint32_t c = S.slot_cfg[g];
    S.cfg_E[c] = recount_energy<BITS>(S.spins + (size_t)c * M.wpc, M);
}

#ifdef REWL_DEBUG_CHECKS
// Debug build, before every window check: the energy each walker keeps
// incrementally must equal a full recount of its configuration (Eq. 2).
template <int BITS>
__global__ void energy_check_kernel(Model M, State S) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M.G || S.done[g / M.m] || *(volatile unsigned int *)&S.ctl->all_done) return;
    const uint32_t c = S.slot_cfg[g];
    if (S.cfg_E[c] != recount_energy<BITS>(S.spins + (size_t)c * M.wpc, M)) atomicOr(&S.ctl->error, ERR_ENERGY);
}
#endif

// ---------------------------------------------------------------------------
size_t sweep_smem_per_walker(const Model &M) {
    return (size_t)M.B * (sizeof(double) + sizeof(uint32_t)) + (size_t)M.wpc * sizeof(uint32_t);
}

SweepPlan plan_sweep(const Model &M, int num_sms, size_t smem_optin, int kind, int lanes, int lat_mode) {
    SweepPlan p{};
    p.kind = kind;
    if (kind == SWEEP_FAST) {
        // lane groups while walkers are few (each walker's chain is what bounds
        // the rate); a thread per walker, state in global memory, once there are
        // enough of them to fill the SMs by themselves (measured crossover on
        // GB300: between 4096 and 16384 walkers)
        // (tiny lattices: 32 proposals of a batch touch each other's neighbourhoods
        // so often that 8-lane trees win -- measured on the L = 8 Ising workload:
        // 2.13e7 flips/s with 8 lanes against 1.74e7 with 32)
        const bool chosen = lanes <= 0;
        if (chosen) lanes = M.G <= 80 * num_sms ? (M.N <= 128 ? 8 : 32) : 1;
        // a window too wide for a lane group's shared memory (its ln g shadow):
        // a thread per walker with the whole state in global memory
        if (chosen && lanes > 1 && lat_mode != 2 &&
            fast_smem_per_walker(M, lanes, M.wpc * 4 > kSharedLatticeMax) > smem_optin)
            lanes = 1;
        p.lanes = lanes;
        p.lat_global = lat_mode == 1   ? 1
                       : lat_mode == 2 ? 0
                                       : ((M.wpc * 4 > kSharedLatticeMax || lanes == 1) ? 1 : 0);
        const size_t per = fast_smem_per_walker(M, lanes, p.lat_global != 0);
        int cap = per ? (int)(smem_optin / per) : 256;  // per = 0: nothing in shared memory
        if (cap > 256 / lanes) cap = 256 / lanes;
        int P = (M.G + num_sms - 1) / num_sms;
        if (P < 1) P = 1;
        if (P > cap) P = cap;
        p.P = P;
        p.threads = ((P * lanes + 31) / 32) * 32;
        p.grid = P > 0 ? (M.G + P - 1) / P : 0;
        p.smem = per * (size_t)P;
        return p;
    }
    p.lanes = 1;
    const size_t per = sweep_smem_per_walker(M);
    int cap = (int)(smem_optin / per);
    if (cap > 256) cap = 256;
    int P = (M.G + num_sms - 1) / num_sms;
    if (P < 1) P = 1;
    if (P > cap) P = cap;
    p.P = P;
    p.threads = ((P + 31) / 32) * 32;
    if (p.threads < 128) p.threads = 128;
    p.grid = P > 0 ? (M.G + P - 1) / P : 0;
    p.smem = per * (size_t)P;
    return p;
}

cudaError_t launch_init(const Model &M, const State &S, cudaStream_t s) {
    const int threads = 64, grid = (M.G + threads - 1) / threads;
    if (M.bits == 8) init_kernel<8><<<grid, threads, 0, s>>>(M, S);
    else init_kernel<4><<<grid, threads, 0, s>>>(M, S);
    return cudaGetLastError();
}

cudaError_t prepare_sweep(const Model &M, const SweepPlan &p) {
    if (p.kind == SWEEP_FAST) return launch_sweep_fast(M, State{}, p, nullptr, true);
    if (M.bits == 8)
        return cudaFuncSetAttribute(sweep_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    return cudaFuncSetAttribute(sweep_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
}

cudaError_t launch_sweep(const Model &M, const State &S, const SweepPlan &p, cudaStream_t s) {
    if (p.kind == SWEEP_FAST) return launch_sweep_fast(M, S, p, s, false);
    if (M.bits == 8) sweep_kernel<8><<<p.grid, p.threads, p.smem, s>>>(M, S, p.P);
    else sweep_kernel<4><<<p.grid, p.threads, p.smem, s>>>(M, S, p.P);
    return cudaGetLastError();
}

cudaError_t launch_window_check(const Model &M, const State &S, cudaStream_t s) {
#ifdef REWL_DEBUG_CHECKS
    if (M.bits == 8) energy_check_kernel<8><<<(M.G + 63) / 64, 64, 0, s>>>(M, S);
    else energy_check_kernel<4><<<(M.G + 63) / 64, 64, 0, s>>>(M, S);
#endif
    window_check_kernel<<<M.h, CHECK_THREADS, 0, s>>>(M, S);
    return cudaGetLastError();
}

cudaError_t launch_exchange(const Model &M, const State &S, cudaStream_t s) {
    exchange_kernel<<<1, XCH_THREADS, 0, s>>>(M, S);
    return cudaGetLastError();
}

cudaError_t launch_count_spins(const Model &M, const State &S, cudaStream_t s) {
    if (M.bits == 8) count_spins_kernel<8><<<M.G, 256, 0, s>>>(M, S);
    else count_spins_kernel<4><<<M.G, 256, 0, s>>>(M, S);
    return cudaGetLastError();
}

cudaError_t launch_production_sweep(const Model &M, const State &S, cudaStream_t s) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    int per = (M.G + sms - 1) / sms;  // walkers per CTA: one CTA per SM
    if (per > 256) per = 256;
    const int threads = ((per + 31) / 32) * 32, grid = (M.G + per - 1) / per;
    if (M.bits == 8) production_kernel<8><<<grid, threads, 0, s>>>(M, S, per);
    else production_kernel<4><<<grid, threads, 0, s>>>(M, S, per);
    return cudaGetLastError();
}

cudaError_t launch_batch_check(const InstDev *inst, const WinItem *wins, int n_wins, cudaStream_t s) {
    if (n_wins <= 0) return cudaSuccess;
    batch_check_kernel<<<n_wins, CHECK_THREADS, 0, s>>>(inst, wins);
    return cudaGetLastError();
}

cudaError_t launch_batch_exchange(const InstDev *inst, int n_inst, cudaStream_t s) {
    if (n_inst <= 0) return cudaSuccess;
    batch_exchange_kernel<<<n_inst, XCH_THREADS, 0, s>>>(inst);
    return cudaGetLastError();
}

cudaError_t launch_get_spins(const Model &M, const State &S, uint8_t *out, cudaStream_t s) {
    const int threads = 256, grid = 256;
    if (M.bits == 8) get_spins_kernel<8><<<grid, threads, 0, s>>>(M, S, out);
    else get_spins_kernel<4><<<grid, threads, 0, s>>>(M, S, out);
    return cudaGetLastError();
}

cudaError_t launch_set_spins(const Model &M, const State &S, const uint8_t *in, cudaStream_t s) {
    const int threads = 256, grid = 256;
    if (M.bits == 8) set_spins_kernel<8><<<grid, threads, 0, s>>>(M, S, in);
    else set_spins_kernel<4><<<grid, threads, 0, s>>>(M, S, in);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int rg = (M.G + 63) / 64;
    if (M.bits == 8) recount_kernel<8><<<rg, 64, 0, s>>>(M, S);
    else recount_kernel<4><<<rg, 64, 0, s>>>(M, S);
    return cudaGetLastError();
}

}  // namespace rewl
