// SVD of the small factor (Eq. i3) and the lift U = Q W (Eq. i4).
//
// B = Q^* A_c is l x n.  The library forms B^* = A_c^* Q (n x l) with the
// adjoint product, factors it as B^* = Q2 R (CholeskyQR), and then needs only
// the SVD of the l x l triangular R^T = W Sigma Z^T, since
// B = R^T Q2^T = W Sigma (Q2 Z)^T.  So U = Q W and V = Q2 Z.
//
// The l x l SVD is one-sided Jacobi (Hestenes; Demmel & Veselic 1992): plane
// rotations applied on the right orthogonalise the columns of M = R^T.  One
// CTA holds M in shared memory (column j of M is row j of R, contiguous) and
// runs the l/2 disjoint rotations of a round-robin step in parallel, four or
// eight lanes per column pair.  The rotations are logged; a second kernel replays
// them on the rows of the identity (every row of Z evolves independently, one
// warp per row), which keeps Z out of the Jacobi CTA's shared memory.
#include "internal.cuh"

#include <algorithm>

namespace rpca {

namespace {

constexpr int kJacThreads = 1024;
constexpr int kMaxSweeps = 40;

__host__ __device__ __forceinline__ int even_up(int l) { return l + (l & 1); }
// row length of the Jacobi CTA's copy of M (16-byte rows for float4 access)
__host__ __device__ __forceinline__ int jac_ldm(int l) { return (l + 3) & ~3; }

// LPP lanes per column pair; CACHE > 0: each lane keeps its CACHE float4 of both
// columns in registers between the inner products and the rotation (ldm / 4 <=
// LPP * CACHE), so that a round reads shared memory once.
template <int LPP, int CACHE>
__global__ void __launch_bounds__(CACHE > 0 ? 512 : kJacThreads)
jacobi_kernel(const float *__restrict__ R, int l, float2 *__restrict__ rot, int *__restrict__ sweeps_out,
              float *__restrict__ sig, int *__restrict__ perm, float *__restrict__ Wk, int lp, int k,
              int kp, DevStatus *__restrict__ st) {
    extern __shared__ float4 Ms4[];    // l rows of ldm floats: row j = column j of M = R^T
    float *Ms = reinterpret_cast<float *>(Ms4);
    const int ldm = jac_ldm(l);        // multiple of 4, columns l..ldm-1 zero
    const int nv = ldm / 4;            // float4 per row
    __shared__ int s_rot;
    __shared__ int s_mu;               // largest predicted next-sweep measure (float bits, >= 0)
    __shared__ float s_sig[RPCA_MAX_L];
    const int tid = threadIdx.x;
    const int L = even_up(l);
    const int npairs = L / 2;

    for (int e = tid; e < l * ldm; e += blockDim.x) {
        const int j = e / ldm, c = e - j * ldm;
        Ms[e] = c < l ? R[(size_t)j * l + c] : 0.f;
    }
    __syncthreads();

    const int g = tid / LPP, lane = tid % LPP;
    const bool live = g < npairs;
    const float tol = 8.0f * sqrtf((float)l) * 0x1p-24f;
    float2 *rlog = rot + g;
    int sweep = 0;
    bool early = false;
    for (; sweep < kMaxSweeps; ++sweep) {
        if (tid == 0) { s_rot = 0; s_mu = 0; }
        __syncthreads();
        // circle-method round robin: positions g and L-1-g; each step moves every
        // player but 0 one place along 1..L-1
        int pa = g == 0 ? 0 : g, pb = L - 1 - g;
        float mu_max = 0.f;
        for (int step = 0; step < L - 1; ++step) {
            const int p = live ? min(pa, pb) : 0, q = live ? max(pa, pb) : 0;
            const bool valid = live && q < l;
            float a0 = 0.f, b0 = 0.f, c0 = 0.f, a1 = 0.f, b1 = 0.f, c1 = 0.f;
            float4 *mp = Ms4 + p * nv, *mq = Ms4 + q * nv;
            float4 xc[CACHE > 0 ? CACHE : 1], yc[CACHE > 0 ? CACHE : 1];
            if (CACHE > 0) {
#pragma unroll
                for (int it = 0; it < CACHE; ++it) {
                    const int e = lane + LPP * it;
                    xc[it] = make_float4(0.f, 0.f, 0.f, 0.f);
                    yc[it] = xc[it];
                    if (valid && e < nv) { xc[it] = mp[e]; yc[it] = mq[e]; }
                }
#pragma unroll
                for (int it = 0; it < CACHE; ++it) {
                    const float4 x = xc[it], y = yc[it];
                    float &a = (it & 1) ? a1 : a0, &b = (it & 1) ? b1 : b0, &c = (it & 1) ? c1 : c0;
                    a = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, a))));
                    b = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, b))));
                    c = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, c))));
                }
            } else if (valid) {
#pragma unroll 2
                for (int e = lane; e < nv; e += LPP) {
                    const float4 x = mp[e], y = mq[e];
                    a0 = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, a0))));
                    b0 = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, b0))));
                    c0 = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, c0))));
                }
            }
            float a = a0 + a1, b = b0 + b1, c = c0 + c1;
#pragma unroll
            for (int off = 1; off < LPP; off <<= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, off);
                b += __shfl_xor_sync(0xffffffffu, b, off);
                c += __shfl_xor_sync(0xffffffffu, c, off);
            }
            // the rotation that zeroes c (Rutishauser's formulas), with fast intrinsics.  The
            // rotations are not exactly orthogonal (cs^2 + sn^2 = 1 to a few ulps, and the
            // error has a sign: over the hundreds of rotations a column takes, the column
            // norms drift by ~1e-5); the replayed Z drifts by the same factors, and
            // svd_finish_kernel divides it out
            float cs = 1.f, sn = 0.f;
            const float mu = valid ? fabsf(c) * rsqrtf(a) * rsqrtf(b) : 0.f;   // NaN when a b = 0
            if (mu > tol) {
                // by quadratic convergence the next sweep's largest measure is bounded by
                // about l mu^2 / delta (the off-diagonal mass of the whole sweep over the
                // relative gap delta of the pair's squared column norms)
                const float delta = fabsf(b - a) / (a + b);
                mu_max = fmaxf(mu_max, delta > 0.f ? fminf((float)l * mu * mu / delta, 1.f) : 1.f);
                const float zeta = __fdividef(b - a, 2.f * c);
                const float t = copysignf(__frcp_rn(fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f))), zeta);
                cs = rsqrtf(fmaf(t, t, 1.f));
                sn = cs * t;
                if (CACHE > 0) {
#pragma unroll
                    for (int it = 0; it < CACHE; ++it) {
                        const int e = lane + LPP * it;
                        const float4 x = xc[it], y = yc[it];
                        if (e < nv) {
                            mp[e] = make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z,
                                                cs * x.w - sn * y.w);
                            mq[e] = make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z,
                                                sn * x.w + cs * y.w);
                        }
                    }
                } else {
#pragma unroll 2
                    for (int e = lane; e < nv; e += LPP) {
                        const float4 x = mp[e], y = mq[e];
                        mp[e] = make_float4(cs * x.x - sn * y.x, cs * x.y - sn * y.y, cs * x.z - sn * y.z,
                                            cs * x.w - sn * y.w);
                        mq[e] = make_float4(sn * x.x + cs * y.x, sn * x.y + cs * y.y, sn * x.z + cs * y.z,
                                            sn * x.w + cs * y.w);
                    }
                }
                s_rot = 1;                       // any rotation this sweep (a flag, not a count)
            }
            if (live && lane == 0) *rlog = make_float2(cs, sn);
            rlog += npairs;
            pa = pa == 0 ? 0 : (pa == L - 1 ? 1 : pa + 1);
            pb = pb == 0 ? 0 : (pb == L - 1 ? 1 : pb + 1);
            __syncthreads();
        }
        // the sweep's largest measure (once per sweep: warp max, one atomic per warp)
#pragma unroll
        for (int off = 16; off; off >>= 1) mu_max = fmaxf(mu_max, __shfl_xor_sync(0xffffffffu, mu_max, off));
        if ((tid & 31) == 0 && mu_max > 0.f) atomicMax(&s_mu, __float_as_int(mu_max));
        __syncthreads();
        if (s_rot == 0) { ++sweep; break; }
        // quadratic convergence: when every rotation's predicted next measure is below
        // tol the next sweep would rotate nothing, so it is not run (pairs of nearly
        // equal column norms, small delta, keep the iteration going longer)
        if (__int_as_float(s_mu) < tol) { ++sweep; early = true; break; }
        __syncthreads();
    }
    // sweep = number of logged sweeps (the last one made no rotation, or every rotation's
    // predicted next measure was below tol, or the cap was hit)
    if (tid == 0) {
        *sweeps_out = sweep;
        st->jacobi_sweeps = sweep;
        if (sweep >= kMaxSweeps && s_rot != 0 && !early) atomicAdd(&st->jacobi_unconverged, 1);
    }

    // singular values = column norms; sort descending (ties by index)
    // (warp-uniform trip count: every lane reaches the full-mask shuffles)
    for (int j0 = 0; j0 < l; j0 += (int)blockDim.x / LPP) {
        const int j = j0 + g;
        float s2 = 0.f;
        if (j < l)
            for (int e = lane; e < l; e += LPP) s2 = fmaf(Ms[j * ldm + e], Ms[j * ldm + e], s2);
        for (int off = 1; off < LPP; off <<= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        if (j < l && lane == 0) s_sig[j] = sqrtf(s2);
    }
    __syncthreads();
    for (int j = tid; j < l; j += blockDim.x) {
        const float sj = s_sig[j];
        int rank = 0;
        for (int i = 0; i < l; ++i) {
            const float si = s_sig[i];
            rank += (si > sj) || (si == sj && i < j);
        }
        perm[rank] = j;
        sig[rank] = sj;
    }
    __syncthreads();
    // Wk[i][r] = M[:, perm[r]][i] / sigma_r  (rows >= l and columns >= k zero)
    for (int e = tid; e < lp * kp; e += blockDim.x) {
        const int i = e / kp, r = e % kp;
        float v = 0.f;
        if (i < l && r < k) {
            const int j = perm[r];
            const float s = s_sig[j];
            v = s > 0.f ? Ms[j * ldm + i] / s : 0.f;
        }
        Wk[e] = v;
    }
}

// Z = product of the logged rotations applied to the identity.  Every row of Z
// evolves independently, so each warp owns one row (in shared memory) and applies
// the rounds in order, lanes taking the disjoint pairs of a round.  The logged
// rotations pass through shared memory kReplayChunk rounds at a time, double
// buffered: the next chunk's loads are in flight while the current one is applied.
// Zk[i][r] = Z[i][perm[r]].
constexpr int kReplayWarps = 8;
constexpr int kReplayChunk = 32;
constexpr int kReplayGroups = (RPCA_MAX_L / 2 + 31) / 32;   // pair groups per lane
constexpr int kReplayPre = (kReplayChunk * (RPCA_MAX_L / 2) + kReplayWarps * 32 - 1) / (kReplayWarps * 32);

__global__ void __launch_bounds__(kReplayWarps * 32)
replay_kernel(const float2 *__restrict__ rot, const int *__restrict__ sweeps_ptr, int l,
              const int *__restrict__ perm, float *__restrict__ Zk, int lp, int k, int kp) {
    __shared__ float Z[kReplayWarps][RPCA_MAX_L + 1];
    extern __shared__ float2 rs[];                            // [2][kReplayChunk][npairs]
    const int L = even_up(l), npairs = L / 2;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int i = blockIdx.x * kReplayWarps + warp;           // this warp's row of Z
    for (int c = lane; c < l; c += 32) Z[warp][c] = (i == c) ? 1.f : 0.f;
    const int rounds = *sweeps_ptr * (L - 1);
    const int nchunks = (rounds + kReplayChunk - 1) / kReplayChunk;
    float2 pre[kReplayPre];
    auto load = [&](int ch) {
        const int c0 = ch * kReplayChunk, n = min(kReplayChunk, rounds - c0) * npairs;
#pragma unroll
        for (int u = 0; u < kReplayPre; ++u) {
            const int e = tid + u * nt;
            pre[u] = e < n ? rot[(size_t)c0 * npairs + e] : make_float2(1.f, 0.f);
        }
    };
    auto store = [&](int ch) {
        const int c0 = ch * kReplayChunk, n = min(kReplayChunk, rounds - c0) * npairs;
        float2 *dst = rs + (size_t)(ch & 1) * kReplayChunk * npairs;
#pragma unroll
        for (int u = 0; u < kReplayPre; ++u) {
            const int e = tid + u * nt;
            if (e < n) dst[e] = pre[u];
        }
    };
    if (nchunks > 0) { load(0); store(0); }
    __syncthreads();
    // positions of this lane's pair groups g = lane + 32 u in the round-robin circle
    int pa[kReplayGroups], pb[kReplayGroups];
    int step = 0;
    for (int ch = 0; ch < nchunks; ++ch) {
        if (ch + 1 < nchunks) load(ch + 1);
        const int nr = min(kReplayChunk, rounds - ch * kReplayChunk);
        const float2 *cur = rs + (size_t)(ch & 1) * kReplayChunk * npairs;
        if (i < l) {
            for (int r = 0; r < nr; ++r, ++step) {
                if (step == L - 1) step = 0;
                if (step == 0) {                      // a new sweep: the circle starts over
#pragma unroll
                    for (int u = 0; u < kReplayGroups; ++u) {
                        const int g = lane + 32 * u;
                        pa[u] = g == 0 ? 0 : g;
                        pb[u] = L - 1 - g;
                    }
                }
#pragma unroll
                for (int u = 0; u < kReplayGroups; ++u) {
                    const int g = lane + 32 * u;
                    const int p = min(pa[u], pb[u]), q = max(pa[u], pb[u]);
                    if (g < npairs && q < l) {
                        const float2 csn = cur[r * npairs + g];
                        const float x = Z[warp][p], y = Z[warp][q];
                        Z[warp][p] = csn.x * x - csn.y * y;
                        Z[warp][q] = csn.y * x + csn.x * y;
                    }
                    pa[u] = pa[u] == 0 ? 0 : (pa[u] == L - 1 ? 1 : pa[u] + 1);
                    pb[u] = pb[u] == 0 ? 0 : (pb[u] == L - 1 ? 1 : pb[u] + 1);
                }
                __syncwarp();
            }
        }
        if (ch + 1 < nchunks) store(ch + 1);
        __syncthreads();
    }
    if (i < lp)
        for (int r = lane; r < kp; r += 32) {
            float v = 0.f;
            if (i < l && r < k) v = Z[warp][perm[r]];
            Zk[(size_t)i * kp + r] = v;
        }
}

// The rotation-norm correction.  The Jacobi's rotations are orthogonal only to a
// few ulps with a systematic sign, so every rotation scales the two columns it
// mixes by the same factor in the rotated M and in the replayed Z (~1e-5 over a
// full SVD at l = 150).  Column r of M J and of Z = J carry the same factor, so
// sigma_r = |(M J)_r| / |Z_r| and Z_r / |Z_r| remove it while W (a direction) is
// unchanged; the one-sided Jacobi's relative accuracy on small singular values is
// kept.  The k triplets are then re-sorted (descending, ties by index).
// One CTA; scratch: 2 lp kp floats (the rotation log, no longer needed after the replay).
constexpr int kFinThreads = 512;

__global__ void __launch_bounds__(kFinThreads)
svd_finish_kernel(int l, int lp, int k, int kp, float *__restrict__ Wk, float *__restrict__ Zk,
                  float *__restrict__ sig, float *__restrict__ scratch) {
    __shared__ float snew[RPCA_MAX_L], inz[RPCA_MAX_L];
    __shared__ int rank_of[RPCA_MAX_L];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
    for (int r = warp; r < k; r += nwarps) {
        float nz = 0.f;
        for (int i = lane; i < l; i += 32) nz = fmaf(Zk[(size_t)i * kp + r], Zk[(size_t)i * kp + r], nz);
#pragma unroll
        for (int off = 16; off; off >>= 1) nz += __shfl_xor_sync(0xffffffffu, nz, off);
        if (lane == 0) {
            const float f = nz > 0.f ? 1.f / sqrtf(nz) : 0.f;
            inz[r] = f;
            snew[r] = nz > 0.f ? sig[r] * f : sig[r];
        }
    }
    __syncthreads();
    for (int r = tid; r < k; r += blockDim.x) {
        const float sr = snew[r];
        int rank = 0;
        for (int q = 0; q < k; ++q) rank += (snew[q] > sr) || (snew[q] == sr && q < r);
        rank_of[r] = rank;
    }
    __syncthreads();
    float *Ws = scratch, *Zs = scratch + (size_t)lp * kp;
    for (int e = tid; e < lp * kp; e += blockDim.x) {
        Ws[e] = Wk[e];
        Zs[e] = Zk[e];
    }
    __syncthreads();
    for (int r = tid; r < k; r += blockDim.x) sig[rank_of[r]] = snew[r];
    for (int e = tid; e < lp * kp; e += blockDim.x) {
        const int i = e / kp, r = e - i * kp;
        if (r < k) {
            const int dst = i * kp + rank_of[r];
            Wk[dst] = Ws[e];
            Zk[dst] = Zs[e] * inz[r];
        }
    }
}

// Per column r < k: flip V[:, r] when its largest-|entry| (first on ties) is
// negative; apply the same sign to Wk[:, r]; S[r] = sig[r].  One CTA per column; each
// thread scans its rows eight at a time (eight strided loads in flight), in increasing
// row order, so "strictly greater" keeps the first index as in a plain scan.
constexpr int kSignThreads = 1024;

__global__ void __launch_bounds__(kSignThreads)
sign_fix_kernel(float *__restrict__ V, int64_t n, int64_t ldv, float *__restrict__ Wk, int lp, int kp,
                const float *__restrict__ sig, float *__restrict__ S) {
    const int r = blockIdx.x;
    const int nt = blockDim.x;
    __shared__ float sv[kSignThreads];
    __shared__ int64_t si[kSignThreads];
    float best = -1.f;
    int64_t bi = 0;
    for (int64_t i0 = threadIdx.x; i0 < n; i0 += 8 * (int64_t)nt) {
        float a[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int64_t i = i0 + (int64_t)u * nt;
            a[u] = i < n ? fabsf(V[i * ldv + r]) : -1.f;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (a[u] > best) { best = a[u]; bi = i0 + (int64_t)u * nt; }   // strictly greater keeps the first index
    }
    sv[threadIdx.x] = best;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int off = nt / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            const float ob = sv[threadIdx.x + off];
            const int64_t oi = si[threadIdx.x + off];
            if (ob > sv[threadIdx.x] || (ob == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = ob;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    const bool flip = n > 0 && V[si[0] * ldv + r] < 0.f;
    __syncthreads();
    if (flip) {
        for (int64_t i = threadIdx.x; i < n; i += nt) V[i * ldv + r] = -V[i * ldv + r];
        for (int i = threadIdx.x; i < lp; i += nt) Wk[(size_t)i * kp + r] = -Wk[(size_t)i * kp + r];
    }
    if (threadIdx.x == 0) S[r] = sig[r];
}

}  // namespace

size_t small_svd_rot_floats(int l) {
    const int L = even_up(l);
    return (size_t)kMaxSweeps * (L - 1) * (L / 2) * 2;
}

int launch_small_svd(const float *R, int l, int lp, int k, int kp, float *Wk, float *Zk, float *sig,
                     float *rot, float *zbuf, int *perm, DevStatus *st, cudaStream_t s) {
    int *sweeps = reinterpret_cast<int *>(zbuf);
    const size_t smem = (size_t)l * jac_ldm(l) * sizeof(float);
    const int smem_max = (int)((size_t)RPCA_MAX_L * jac_ldm(RPCA_MAX_L) * sizeof(float));
    // Eight lanes per column pair.  l <= 128 (at most 32 float4 per column): each lane
    // keeps four float4 of both columns in registers; wider: columns re-read.  (Four
    // lanes per pair with eight float4 each, half as many warps, measured 0.80 against
    // 0.70 ms per small SVD at l = 102.)
    const bool cached = jac_ldm(l) / 4 <= 8 * 4;
    auto kern = cached ? jacobi_kernel<8, 4> : jacobi_kernel<8, 0>;
    const int lpp = 8;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max) != cudaSuccess)
        return RPCA_ERR_CUDA;
    // lpp lanes per column pair of a round; no idle warps at the round barriers
    const int threads = (int)std::min<int64_t>(cached ? 512 : kJacThreads,
                                               std::max<int64_t>(64, round_up(lpp * (even_up(l) / 2), 32)));
    kern<<<1, threads, smem, s>>>(R, l, reinterpret_cast<float2 *>(rot), sweeps, sig, perm, Wk, lp, k, kp, st);
    RPCA_CHECK_LAUNCH();
    const int grid = (int)cdiv(lp, kReplayWarps);
    const size_t rsmem = (size_t)2 * kReplayChunk * (even_up(l) / 2) * sizeof(float2);
    if (cudaFuncSetAttribute(replay_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)((size_t)2 * kReplayChunk * (RPCA_MAX_L / 2) * sizeof(float2))) != cudaSuccess)
        return RPCA_ERR_CUDA;
    replay_kernel<<<grid, kReplayWarps * 32, rsmem, s>>>(reinterpret_cast<const float2 *>(rot), sweeps, l, perm, Zk,
                                                         lp, k, kp);
    RPCA_CHECK_LAUNCH();
    svd_finish_kernel<<<1, kFinThreads, 0, s>>>(l, lp, k, kp, Wk, Zk, sig, rot);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

int launch_sign_fix(float *V, int64_t n, int64_t ldv, int k, float *Wk, int lp, int kp,
                    const float *sig, float *S, cudaStream_t s) {
    sign_fix_kernel<<<k, kSignThreads, 0, s>>>(V, n, ldv, Wk, lp, kp, sig, S);
    RPCA_CHECK_LAUNCH();
    return RPCA_OK;
}

}  // namespace rpca
