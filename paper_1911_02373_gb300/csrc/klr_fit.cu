// F1-F4: batched rational fits (Section V-E; Section IV, step 2).
//
// One warp per fit.  The fit's samples are streamed once from HBM (coalesced,
// 32 samples per step, staged as powers of the scaled coordinates in shared
// memory) while the warp accumulates the moment sums
//     M_k[mu] = sum_s y_s^k x_s^mu,  k = 0, 1, 2,  deg(mu) <= 2d,
// which determine every entry of the Gram matrix G = A^T A of
// A = [Phi | -y Phi]:  G_pp[i][j] = M_0[mu_i + mu_j],
// G_pq[i][j] = -M_1[mu_i + mu_j], G_qq[i][j] = M_2[mu_i + mu_j].
// The moments are about half the multiply-adds of a direct Gram at degree 2
// and a third at degree 3.  Lanes split the work as (sample group x moment
// group) so each lane keeps only a few accumulators in registers.
//
// The small solve is FP64: power-of-two column equilibration from the Gram
// diagonal, shifted Cholesky factorisation and inverse iteration for the
// smallest eigenpair (the smallest right singular vector of A D), a second
// shift close below the Rayleigh quotient when the fit is noisy, deflated
// inverse iteration for the next eigenvalue (rank test), and optional
// refinement passes that recompute A^T A v from the samples in FP64 and take a
// preconditioned inverse-iteration step (Knyazev-Neymeyr PINVIT) with the
// Cholesky factor as preconditioner.
#include <cfloat>
#include <type_traits>

#include "klr_common.cuh"

namespace klr {

namespace {

constexpr int kMG = 16;                 // lanes sharing one sample (moment groups)
constexpr int kSG = 32 / kMG;           // sample groups per warp
constexpr int kRefineMaxU = 40;         // unknowns supported by refinement passes

enum { ACC_FP64 = 0, ACC_DF32 = 1, ACC_FP32 = 2 };

struct FitParams {
    int n_fits, n_vars, degree, m, u, n_mom;
    int n_scale_log2, b_scale_log2;
    const int64_t* offsets;
    const void* x;
    int64_t x_stride;
    const void* y;
    void* coef;
    int coef_f64;
    int32_t* status;
    double* diag;
    int refine;
    int ld;        // leading dimension of the Gram matrix in shared memory
    int warp_smem; // bytes of shared memory per warp
    uint8_t exps[kMaxMoments][kMaxVars];
    uint8_t pair[kMaxBasis][kMaxBasis];
};

__device__ __forceinline__ bool is_pow2_positive(float v) {
    unsigned b = __float_as_uint(v);
    return (b & 0x007FFFFFu) == 0u && (b >> 23) != 0u && (b >> 31) == 0u;
}
__device__ __forceinline__ bool is_pow2_positive(double v) {
    unsigned long long b = __double_as_longlong(v);
    return (b & 0x000FFFFFFFFFFFFFull) == 0ull && (b >> 52) != 0ull && (b >> 63) == 0ull;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Cholesky of (Ghat - shift I) into the lower triangle of G (leading dim ld);
// the strict upper triangle keeps Ghat, gdiag its diagonal.  Warp-cooperative.
__device__ bool warp_cholesky(double* G, const double* gdiag, int u, int ld, double shift) {
    const int lane = lane_id();
    for (int idx = lane; idx < u * u; idx += 32) {
        int i = idx / u, j = idx % u;
        if (i > j) G[i * ld + j] = G[j * ld + i];
        else if (i == j) G[i * ld + i] = gdiag[i] - shift;
    }
    __syncwarp();
    for (int k = 0; k < u; ++k) {
        double akk = G[k * ld + k];
        if (!(akk > 0.0)) return false;   // uniform across the warp
        double lkk = sqrt(akk);
        for (int i = k + 1 + lane; i < u; i += 32) G[i * ld + k] /= lkk;
        __syncwarp();
        if (lane == 0) G[k * ld + k] = lkk;
        for (int i = k + 1 + lane; i < u; i += 32) {
            double lik = G[i * ld + k];
            for (int j = k + 1; j <= i; ++j) G[i * ld + j] -= lik * G[j * ld + k];
        }
        __syncwarp();
    }
    return true;
}

// Solve (L L^T) w = b in place (w holds b on entry).
__device__ void warp_chol_solve(const double* G, int u, int ld, double* w) {
    const int lane = lane_id();
    for (int k = 0; k < u; ++k) {
        double yk = w[k] / G[k * ld + k];
        __syncwarp();
        for (int i = k + 1 + lane; i < u; i += 32) w[i] -= G[i * ld + k] * yk;
        if (lane == 0) w[k] = yk;
        __syncwarp();
    }
    for (int k = u - 1; k >= 0; --k) {
        double xk = w[k] / G[k * ld + k];
        __syncwarp();
        for (int i = lane; i < k; i += 32) w[i] -= G[k * ld + i] * xk;
        if (lane == 0) w[k] = xk;
        __syncwarp();
    }
}

// y = Ghat v (Ghat in the strict upper triangle + gdiag).
__device__ void warp_gram_matvec(const double* G, const double* gdiag, int u, int ld,
                                 const double* v, double* y) {
    const int lane = lane_id();
    for (int i = lane; i < u; i += 32) {
        double acc = gdiag[i] * v[i];
        for (int j = 0; j < u; ++j)
            if (j != i) acc += G[min(i, j) * ld + max(i, j)] * v[j];
        y[i] = acc;
    }
    __syncwarp();
}

__device__ double warp_dot(const double* a, const double* b, int u) {
    double s = 0.0;
    for (int i = lane_id(); i < u; i += 32) s += a[i] * b[i];
    return warp_sum(s);
}

__device__ void warp_scale(double* a, int u, double s) {
    for (int i = lane_id(); i < u; i += 32) a[i] *= s;
    __syncwarp();
}

// w <- w - (w.v) v, then normalise.  Returns the norm before normalising.
__device__ double warp_orth_normalise(double* w, const double* v, int u, bool orth) {
    if (orth) {
        double c = warp_dot(w, v, u);
        for (int i = lane_id(); i < u; i += 32) w[i] -= c * v[i];
        __syncwarp();
    }
    double n = sqrt(warp_dot(w, w, u));
    if (n > 0.0) warp_scale(w, u, 1.0 / n);
    __syncwarp();
    return n;
}

__device__ void warp_copy(double* dst, const double* src, int u) {
    for (int i = lane_id(); i < u; i += 32) dst[i] = src[i];
    __syncwarp();
}

template <typename TS, int ACC, int MAXT>
__global__ void __launch_bounds__(128)
fit_kernel(const __grid_constant__ FitParams P) {
    using TC = typename std::conditional<ACC == ACC_FP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = lane_id();
    const int wib = threadIdx.x >> 5;
    const int f = blockIdx.x * (blockDim.x >> 5) + wib;
    if (f >= P.n_fits) return;
    unsigned char* wsm = smem_raw + (size_t)wib * P.warp_smem;

    const int nv = P.n_vars, d = P.degree, m = P.m, u = P.u, n_mom = P.n_mom, ld = P.ld;
    const int PW = 2 * d + 1;              // powers 0..2d per variable
    const int REC = nv * PW + 3;           // powers + (y, y^2 hi, y^2 lo)
    TC* stage = reinterpret_cast<TC*>(wsm);
    double* mom = reinterpret_cast<double*>(wsm + ((32 * REC * sizeof(TC) + 15) & ~15));
    double* G = mom + 3 * n_mom;
    double* gdiag = G + u * ld;
    double* D = gdiag + u;
    double* v = D + u;
    double* w = v + u;
    double* t = w + u;

    const int64_t s0 = P.offsets[f], s1 = P.offsets[f + 1];
    const TS* X = reinterpret_cast<const TS*>(P.x);
    const TS* Y = reinterpret_cast<const TS*>(P.y);
    const double n_scale = ldexp(1.0, -P.n_scale_log2);
    const double b_scale = ldexp(1.0, -P.b_scale_log2);

    // ---- F1 + F2: stream samples, accumulate moments ------------------------
    const int mg = lane % kMG, sg = lane / kMG;
    int off[MAXT][kMaxVars];
    int my_n = 0;
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
        int mu = mg + kMG * i;
        if (mu < n_mom) my_n = i + 1;
#pragma unroll
        for (int vv = 0; vv < kMaxVars; ++vv)
            off[i][vv] = (mu < n_mom && vv < nv) ? vv * PW + P.exps[mu][vv] : 0;
    }
    TC a0[MAXT], a1[MAXT], a2[MAXT];
    float c0[MAXT], c1[MAXT], c2[MAXT];
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
        a0[i] = a1[i] = a2[i] = TC(0);
        c0[i] = c1[i] = c2[i] = 0.f;
    }
    bool bad = false, inexact = false;
    for (int64_t base = s0; base < s1; base += 32) {
        const int64_t s = base + lane;
        if (s < s1) {
            TC* r = stage + lane * REC;
            for (int vv = 0; vv < nv; ++vv) {
                TS raw = X[(int64_t)vv * P.x_stride + s];
                bad |= !isfinite((double)raw);
                if constexpr (ACC == ACC_DF32) inexact |= !is_pow2_positive(raw);
                TC xv = (TC)((double)raw * (vv == 0 ? n_scale : b_scale));
                TC p = TC(1);
                for (int k = 0; k < PW; ++k) {
                    r[vv * PW + k] = p;
                    p *= xv;
                }
            }
            TS yraw = Y[s];
            bad |= !isfinite((double)yraw);
            TC yv = (TC)yraw;
            TC y2h = yv * yv;
            TC y2l = TC(0);
            if constexpr (ACC != ACC_FP64) y2l = fmaf(yv, yv, -y2h);
            r[nv * PW + 0] = yv;
            r[nv * PW + 1] = y2h;
            r[nv * PW + 2] = y2l;
        }
        __syncwarp();
        const int nvalid = (int)min((int64_t)32, s1 - base);
        for (int ts = sg; ts < nvalid; ts += kSG) {
            const TC* r = stage + ts * REC;
            const TC yv = r[nv * PW + 0], y2h = r[nv * PW + 1], y2l = r[nv * PW + 2];
#pragma unroll
            for (int i = 0; i < MAXT; ++i) {
                if (i < my_n) {
                    TC xm = r[off[i][0]] * r[off[i][1]];
                    if (nv > 2) xm *= r[off[i][2]];
                    if (nv > 3) xm *= r[off[i][3]];
                    if constexpr (ACC == ACC_FP64) {
                        a0[i] += xm;
                        a1[i] = fma(yv, xm, a1[i]);
                        a2[i] = fma(y2h, xm, a2[i]);
                    } else if constexpr (ACC == ACC_DF32) {
                        // products of a value and a power of two are exact
                        df_add(a0[i], c0[i], xm);
                        df_add(a1[i], c1[i], yv * xm);
                        df_add(a2[i], c2[i], y2h * xm);
                        c2[i] = fmaf(y2l, xm, c2[i]);
                    } else {
                        a0[i] += xm;
                        a1[i] = fmaf(yv, xm, a1[i]);
                        a2[i] = fmaf(y2h, xm, a2[i]);
                    }
                }
            }
        }
        __syncwarp();
    }
    // reduce across sample groups (lanes mg, mg + 16)
#pragma unroll
    for (int i = 0; i < MAXT; ++i) {
#pragma unroll
        for (int o = kMG; o < 32; o <<= 1) {
            if constexpr (ACC == ACC_DF32) {
                float h, e;
                float oh0 = __shfl_xor_sync(0xffffffffu, a0[i], o);
                float ol0 = __shfl_xor_sync(0xffffffffu, c0[i], o);
                two_sum(a0[i], oh0, h, e);
                a0[i] = h; c0[i] = c0[i] + ol0 + e;
                float oh1 = __shfl_xor_sync(0xffffffffu, a1[i], o);
                float ol1 = __shfl_xor_sync(0xffffffffu, c1[i], o);
                two_sum(a1[i], oh1, h, e);
                a1[i] = h; c1[i] = c1[i] + ol1 + e;
                float oh2 = __shfl_xor_sync(0xffffffffu, a2[i], o);
                float ol2 = __shfl_xor_sync(0xffffffffu, c2[i], o);
                two_sum(a2[i], oh2, h, e);
                a2[i] = h; c2[i] = c2[i] + ol2 + e;
            } else {
                a0[i] += __shfl_xor_sync(0xffffffffu, a0[i], o);
                a1[i] += __shfl_xor_sync(0xffffffffu, a1[i], o);
                a2[i] += __shfl_xor_sync(0xffffffffu, a2[i], o);
            }
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    inexact = __any_sync(0xffffffffu, inexact);
    if (sg == 0) {
#pragma unroll
        for (int i = 0; i < MAXT; ++i) {
            if (i < my_n) {
                int mu = mg + kMG * i;
                mom[mu] = (double)a0[i] + (ACC == ACC_DF32 ? (double)c0[i] : 0.0);
                mom[n_mom + mu] = (double)a1[i] + (ACC == ACC_DF32 ? (double)c1[i] : 0.0);
                mom[2 * n_mom + mu] = (double)a2[i] + (ACC == ACC_DF32 ? (double)c2[i] : 0.0);
            }
        }
    }
    __syncwarp();

    const int64_t S = s1 - s0;
    int32_t status = 0;
    if (S == 0) status = KLR_FIT_EMPTY;
    else if (bad) status = KLR_FIT_NONFINITE;
    if (status) {
        for (int j = lane; j < u; j += 32) {
            if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = 0.0;
            else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = 0.f;
        }
        if (lane == 0) {
            P.status[f] = status;
            if (P.diag) for (int k = 0; k < 4; ++k) P.diag[(int64_t)f * 4 + k] = 0.0;
        }
        return;
    }
    if (inexact) status |= KLR_FIT_INEXACT;

    // ---- assemble the Gram matrix (upper triangle + diagonal) ---------------
    for (int idx = lane; idx < u * u; idx += 32) {
        int i = idx / u, j = idx % u;
        if (j < i) continue;
        int bi = i >= m, bj = j >= m;
        double val = mom[(bi + bj) * n_mom + P.pair[i - bi * m][j - bj * m]];
        if (bi != bj) val = -val;
        if (i == j) gdiag[i] = val;
        else G[i * ld + j] = val;
    }
    __syncwarp();
    // power-of-two equilibration: D_j = 2^-floor(e_j / 2), e_j = frexp exponent of G_jj
    for (int j = lane; j < u; j += 32) {
        double g = gdiag[j];
        double dj = 1.0;
        if (g > 0.0) {
            int e;
            frexp(g, &e);
            dj = ldexp(1.0, -(e >> 1));
        }
        D[j] = dj;
    }
    __syncwarp();
    for (int idx = lane; idx < u * u; idx += 32) {
        int i = idx / u, j = idx % u;
        if (j < i) continue;
        if (i == j) gdiag[i] *= D[i] * D[i];
        else G[i * ld + j] *= D[i] * D[j];
    }
    __syncwarp();
    double trace = 0.0;
    for (int i = lane; i < u; i += 32) trace += gdiag[i];
    trace = warp_sum(trace);

    // ---- F3: smallest eigenpair by shifted inverse iteration ----------------
    const double eps = DBL_EPSILON;
    const double jitter = 4.0 * u * eps * trace;
    double shift = -jitter;                       // factor Ghat + jitter I
    bool ok = warp_cholesky(G, gdiag, u, ld, shift);
    if (!ok) {
        shift = -1024.0 * jitter;
        ok = warp_cholesky(G, gdiag, u, ld, shift);
    }
    if (!ok) {
        status |= KLR_FIT_SOLVE_FAILED;
    }
    for (int i = lane; i < u; i += 32) v[i] = 1.0 + 0.0625 * (double)((i * 7) % 11);
    __syncwarp();
    warp_orth_normalise(v, v, u, false);
    double theta = 0.0;
    if (ok) {
        for (int it = 0; it < 3; ++it) {
            warp_chol_solve(G, u, ld, v);
            warp_orth_normalise(v, v, u, false);
        }
        warp_gram_matvec(G, gdiag, u, ld, v, t);
        theta = warp_dot(v, t, u);
        if (theta > 64.0 * u * eps * trace) {
            // A noisy fit: the smallest eigenvalue is well above round-off.  Each
            // round factors Ghat - sigma I for the largest sigma of a ladder
            // below the Rayleigh quotient that keeps the matrix positive
            // definite (so sigma < lambda_min), then iterates; the quotient
            // moves down toward lambda_min and the next round's shift closer.
            const double ladder[8] = {1.0 - 1.0 / 64, 1.0 - 1.0 / 32, 1.0 - 1.0 / 16,
                                      1.0 - 1.0 / 8, 1.0 - 1.0 / 4, 0.5, 0.25, 0.0};
            for (int round = 0; round < 3 && ok; ++round) {
                bool ok2 = false;
                for (int k = 0; k < 8 && !ok2; ++k) {
                    shift = k < 7 ? theta * ladder[k] : -jitter;
                    ok2 = warp_cholesky(G, gdiag, u, ld, shift);
                }
                if (!ok2) {
                    status |= KLR_FIT_SOLVE_FAILED;
                    ok = false;
                    break;
                }
                for (int it = 0; it < 4; ++it) {
                    warp_chol_solve(G, u, ld, v);
                    warp_orth_normalise(v, v, u, false);
                }
                warp_gram_matvec(G, gdiag, u, ld, v, t);
                theta = warp_dot(v, t, u);
            }
        }
    }
    // next-smallest eigenvalue: deflated inverse iteration (rank test)
    double theta2 = 0.0;
    if (ok) {
        for (int i = lane; i < u; i += 32) w[i] = 1.0 + 0.03125 * (double)((i * 5) % 13) - 0.5 * (i & 1);
        __syncwarp();
        warp_orth_normalise(w, v, u, true);
        for (int it = 0; it < 3; ++it) {
            warp_chol_solve(G, u, ld, w);
            warp_orth_normalise(w, v, u, true);
        }
        warp_gram_matvec(G, gdiag, u, ld, w, t);
        theta2 = warp_dot(w, t, u);
        if (theta2 <= 64.0 * u * eps * trace) status |= KLR_FIT_RANK_DEFICIENT;
    }

    // ---- F4: FP64 refinement passes over the samples --------------------------
    int passes = 0;
    if (ok && P.refine > 0 && u <= kRefineMaxU) {
        for (int pass = 0; pass < P.refine; ++pass) {
            constexpr int HM = kRefineMaxU / 2;
            double gp[HM], gq[HM];
#pragma unroll
            for (int j = 0; j < HM; ++j) gp[j] = gq[j] = 0.0;
            for (int64_t s = s0 + lane; s < s1; s += 32) {
                double xs[kMaxVars];
                for (int vv = 0; vv < nv; ++vv)
                    xs[vv] = (double)X[(int64_t)vv * P.x_stride + s] * (vv == 0 ? n_scale : b_scale);
                const double ys = (double)Y[s];
                double ap[HM], aq[HM];
                double r = 0.0;
#pragma unroll
                for (int j = 0; j < HM; ++j) {
                    ap[j] = aq[j] = 0.0;
                    if (j < m) {
                        double p = 1.0;
                        for (int vv = 0; vv < nv; ++vv)
                            for (int e = 0; e < P.exps[j][vv]; ++e) p *= xs[vv];
                        ap[j] = D[j] * p;               // equilibrated row of A
                        aq[j] = -D[m + j] * ys * p;
                        r = fma(ap[j], v[j], r);
                        r = fma(aq[j], v[m + j], r);
                    }
                }
#pragma unroll
                for (int j = 0; j < HM; ++j) {
                    gp[j] = fma(r, ap[j], gp[j]);
                    gq[j] = fma(r, aq[j], gq[j]);
                }
            }
            // reduce across lanes; lane 0 writes t = (A D)^T (A D) v
#pragma unroll
            for (int j = 0; j < HM; ++j) {
                if (j < m) {
                    double sp = warp_sum(gp[j]);
                    double sq = warp_sum(gq[j]);
                    if (lane == 0) {
                        t[j] = sp;
                        t[m + j] = sq;
                    }
                }
            }
            __syncwarp();
            theta = warp_dot(v, t, u);
            // residual r = A^T A v - theta v; correction w = (Ghat - shift)^-1 r, orthogonal to v
            for (int i = lane; i < u; i += 32) w[i] = t[i] - theta * v[i];
            __syncwarp();
            warp_chol_solve(G, u, ld, w);
            double c = warp_dot(w, v, u);
            for (int i = lane; i < u; i += 32) v[i] -= w[i] - c * v[i];
            __syncwarp();
            warp_orth_normalise(v, v, u, false);
            ++passes;
        }
    }

    // ---- coefficients: c = D v, unit norm, sign rule --------------------------
    for (int i = lane; i < u; i += 32) w[i] = D[i] * v[i];
    __syncwarp();
    double nrm = sqrt(warp_dot(w, w, u));
    double sgn = 1.0;
    {
        double q0 = w[m] / nrm;
        if (fabs(q0) >= 1e-12) {
            sgn = q0 > 0.0 ? 1.0 : -1.0;
        } else {
            // largest-magnitude denominator coefficient (first on ties) positive
            double best = -1.0;
            int bi = m;
            for (int j = m; j < u; ++j)
                if (fabs(w[j]) > best) { best = fabs(w[j]); bi = j; }
            sgn = w[bi] > 0.0 ? 1.0 : -1.0;
        }
    }
    const double scale = ok ? sgn / nrm : 0.0;
    for (int j = lane; j < u; j += 32) {
        double cj = w[j] * scale;
        if (P.coef_f64) reinterpret_cast<double*>(P.coef)[(int64_t)f * u + j] = cj;
        else reinterpret_cast<float*>(P.coef)[(int64_t)f * u + j] = (float)cj;
    }
    if (lane == 0) {
        P.status[f] = status;
        if (P.diag) {
            double* dg = P.diag + (int64_t)f * 4;
            dg[0] = trace > 0 ? theta / trace : 0.0;
            dg[1] = trace > 0 ? theta2 / trace : 0.0;
            dg[2] = sqrt(fmax(theta, 0.0) / (double)S) / nrm;
            dg[3] = (double)passes;
        }
    }
}

template <typename TS, int ACC>
klr_status launch_fit(const FitParams& P, int maxt, size_t smem_block, int wpb,
                      cudaStream_t stream) {
    const int blocks = (P.n_fits + wpb - 1) / wpb;
    if (maxt <= 6) {
        auto k = fit_kernel<TS, ACC, 6>;
        KLR_CHECK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_block));
        k<<<blocks, wpb * 32, smem_block, stream>>>(P);
    } else {
        auto k = fit_kernel<TS, ACC, 14>;
        KLR_CHECK_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_block));
        k<<<blocks, wpb * 32, smem_block, stream>>>(P);
    }
    KLR_CHECK_CUDA(cudaGetLastError());
    return KLR_OK;
}

}  // namespace
}  // namespace klr

using namespace klr;

extern "C" klr_status klr_fit(klr_ctx* ctx, const klr_fit_batch* b, void* coef_out,
                              int32_t coef_dtype, int32_t* fit_status, double* fit_diag,
                              void* stream_) {
    KLR_REQUIRE(ctx && b, "klr_fit: NULL context or batch");
    Context* c = reinterpret_cast<Context*>(ctx);
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
    KLR_REQUIRE(b->n_fits >= 0, "klr_fit: n_fits < 0");
    KLR_REQUIRE(b->n_vars == 3 || b->n_vars == 4, "klr_fit: n_vars %d not 3 or 4", b->n_vars);
    KLR_REQUIRE(b->degree >= 1 && b->degree <= 3, "klr_fit: degree %d not in 1..3", b->degree);
    KLR_REQUIRE(b->sample_dtype == KLR_F32 || b->sample_dtype == KLR_F64,
                "klr_fit: bad sample_dtype");
    KLR_REQUIRE(coef_dtype == KLR_F32 || coef_dtype == KLR_F64, "klr_fit: bad coef_dtype");
    KLR_REQUIRE(b->precision >= KLR_FIT_FP64 && b->precision <= KLR_FIT_BF16,
                "klr_fit: bad precision %d", b->precision);
    KLR_REQUIRE(b->refine_iters >= 0 && b->refine_iters <= 8, "klr_fit: refine_iters not in 0..8");
    KLR_REQUIRE(b->n_scale_log2 >= -64 && b->n_scale_log2 <= 64 &&
                b->b_scale_log2 >= -64 && b->b_scale_log2 <= 64, "klr_fit: scale out of range");
    if (b->n_fits == 0) return KLR_OK;
    KLR_REQUIRE(b->offsets && b->x && b->y && coef_out && fit_status,
                "klr_fit: NULL device array");
    KLR_REQUIRE(b->x_stride >= 0, "klr_fit: x_stride < 0");
    if (b->precision == KLR_FIT_DF32)
        KLR_REQUIRE(b->sample_dtype == KLR_F32, "klr_fit: DF32 needs KLR_F32 samples");
    if (b->precision == KLR_FIT_TF32 || b->precision == KLR_FIT_BF16) {
        set_error("klr_fit: tensor-core precision modes are not built in this library");
        return KLR_ENOTSUP;
    }
    Basis basis;
    KLR_REQUIRE(make_basis(b->n_vars, b->degree, &basis), "klr_fit: no basis");
    const int m = basis.m, u = 2 * m;
    if (b->refine_iters > 0 && u > kRefineMaxU) {
        set_error("klr_fit: refinement supports at most %d unknowns (have %d)", kRefineMaxU, u);
        return KLR_ENOTSUP;
    }
    KLR_CHECK_CUDA(cudaSetDevice(c->device));

    FitParams P;
    P.n_fits = b->n_fits;
    P.n_vars = b->n_vars;
    P.degree = b->degree;
    P.m = m;
    P.u = u;
    P.n_mom = basis.n_mom;
    P.n_scale_log2 = b->n_scale_log2;
    P.b_scale_log2 = b->b_scale_log2;
    P.offsets = b->offsets;
    P.x = b->x;
    P.x_stride = b->x_stride;
    P.y = b->y;
    P.coef = coef_out;
    P.coef_f64 = coef_dtype == KLR_F64;
    P.status = fit_status;
    P.diag = fit_diag;
    P.refine = b->refine_iters;
    P.ld = (u % 2) ? u : u + 1;
    memcpy(P.exps, basis.exps, sizeof(P.exps));
    memcpy(P.pair, basis.pair, sizeof(P.pair));

    const bool acc64 = b->precision == KLR_FIT_FP64;
    const size_t tc = acc64 ? 8 : 4;
    const int REC = b->n_vars * (2 * b->degree + 1) + 3;
    size_t per_warp = ((32 * REC * tc + 15) & ~(size_t)15) +
                      sizeof(double) * (3 * basis.n_mom + (size_t)u * P.ld + 6 * u);
    per_warp = (per_warp + 15) & ~(size_t)15;
    P.warp_smem = (int)per_warp;
    int wpb = 4;
    while (wpb > 1 && per_warp * wpb > 96 * 1024) wpb >>= 1;
    if (per_warp * wpb > c->smem_optin) {
        set_error("klr_fit: %zu bytes of shared memory per warp exceed the device limit",
                  per_warp);
        return KLR_ENOTSUP;
    }
    const int maxt = (basis.n_mom + kMG - 1) / kMG;
    const size_t smem_block = per_warp * wpb;
    const bool s64 = b->sample_dtype == KLR_F64;
    switch (b->precision) {
        case KLR_FIT_FP64:
            return s64 ? launch_fit<double, ACC_FP64>(P, maxt, smem_block, wpb, stream)
                       : launch_fit<float, ACC_FP64>(P, maxt, smem_block, wpb, stream);
        case KLR_FIT_DF32:
            return launch_fit<float, ACC_DF32>(P, maxt, smem_block, wpb, stream);
        case KLR_FIT_FP32:
            return s64 ? launch_fit<double, ACC_FP32>(P, maxt, smem_block, wpb, stream)
                       : launch_fit<float, ACC_FP32>(P, maxt, smem_block, wpb, stream);
        default:
            set_error("klr_fit: unsupported precision");
            return KLR_ENOTSUP;
    }
}
