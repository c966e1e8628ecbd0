// lpb_check.cu -- what runs every check_every iterations, all in FP64:
//   the fixed-point residual r = ||T(z) - z||_M (Sec. 4, Eq. residual),
//   relative KKT residuals at T(z) in the original space (Eq. stopping),
//   infeasibility certificates (Eq. primal-infeas, dual-infeas),
//   the batch-averaged restart test and primal-weight update (Sec. 4
//   "Restarts", "Step-size and primal weight"; Sec. 5 "Restarts"),
//   and, between checks, extraction of finished LPs and compaction of the
//   batch (Sec. 5 "Stopping criteria and infeasibility detection").
// Per-LP sums are reduced in a fixed order (per-block partials, then a
// fixed tree), so a solve is bitwise reproducible.
#include <type_traits>

#include "lpb_internal.h"

namespace lpb {

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Vec;
template <> struct Vec<float> { static constexpr int V = 4; };
template <> struct Vec<double> { static constexpr int V = 2; };
template <> struct Vec<dfloat> { static constexpr int V = 2; };

__device__ __forceinline__ void ldg_d(const double* p, double (&r)[2]) {
    double2 u = __ldg(reinterpret_cast<const double2*>(p));
    r[0] = u.x; r[1] = u.y;
}
__device__ __forceinline__ void st_d(double* p, const double (&r)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(r[0], r[1]);
}

__device__ __forceinline__ double proj_box(double v, double a, double b) {
    double t = v < b ? v : b;
    return t > a ? t : a;
}
// barrier cone B_[a,b] (Sec. 3)
__device__ __forceinline__ double proj_barrier(double v, double a, double b) {
    const bool li = isinf(a), hi = isinf(b);
    if (li && hi) return 0.0;
    if (li) return v > 0.0 ? v : 0.0;
    if (hi) return v < 0.0 ? v : 0.0;
    return v;
}
// Reduced cost robust to large finite bounds (Sec. 4, stopping criteria;
// the variant of PDLP's Appendix A): v pairs with b when positive and with a
// when negative, and is kept only where that bound is finite and
// |x - bound| <= |x|; elsewhere it is 0 and stays in the dual residual.
__device__ __forceinline__ double robust_rc(double v, double x, double a, double b) {
    if (v > 0.0) return !isinf(b) && fabs(x - b) <= fabs(x) ? v : 0.0;
    if (v < 0.0) return !isinf(a) && fabs(x - a) <= fabs(x) ? v : 0.0;
    return 0.0;
}
// recession cone R_[a,b]; free where both bounds are infinite
__device__ __forceinline__ double proj_recession(double v, double a, double b) {
    const bool li = isinf(a), hi = isinf(b);
    if (li && hi) return v;
    if (hi) return v > 0.0 ? v : 0.0;
    if (li) return v < 0.0 ? v : 0.0;
    return 0.0;
}
// one term of phi_[a,b](v) = b v_+ + a v_-, with 0 * inf = 0
__device__ __forceinline__ double support(double v, double a, double b) {
    if (v > 0.0) return b * v;
    if (v < 0.0) return a * v;
    return 0.0;
}

// ---------------------------------------------------------------------------
// FP64 SpMM of one sparse matrix against two dense operands at once
// ---------------------------------------------------------------------------
template <typename TX>
struct SpmmArgs {
    int rows;
    const int* rp;
    const int* ci;
    const double* va;
    const int* long_rows;
    int n_long, long_thr;
    const TX* s0;
    const TX* s1;
    const TX* s2;
    double* o0;
    double* o1;
    double* o2;
    int ld, ncol;
};

// NOPS = 2: (s0, s1) -> (o0, o1); NOPS = 3 adds s2 -> o2
template <typename TX, int G, int NOPS>
__global__ void __launch_bounds__(kBlock) k_spmm64(const SpmmArgs<TX> a) {
    constexpr int V = Vec<TX>::V, GPB = kBlock / G, TN = G * V;
    __shared__ double red[kBlock * V * NOPS];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int col0 = blockIdx.y * TN + lane * V;
    const bool active = col0 < a.ncol;
    const bool is_long = (int)blockIdx.x < a.n_long;
    int row, slot = 0, nslot = 1;
    if (is_long) {
        row = a.long_rows[blockIdx.x];
        slot = grp;
        nslot = GPB;
    } else {
        row = ((int)blockIdx.x - a.n_long) * GPB + grp;
        if (row >= a.rows) return;
        if (a.rp[row + 1] - a.rp[row] > a.long_thr) return;
    }
    double acc[NOPS][V];
#pragma unroll
    for (int q = 0; q < NOPS; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[q][v] = 0.0;
    const TX* src[3] = {a.s0, a.s1, a.s2};
    if (active) {
        const int end = a.rp[row + 1];
        for (int e = a.rp[row] + slot; e < end; e += nslot) {
            const int c = a.ci[e];
            const double w = a.va[e];
#pragma unroll
            for (int q = 0; q < NOPS; ++q) {
                double x[V];
                ldg_d(src[q] + (size_t)c * a.ld + col0, x);
#pragma unroll
                for (int v = 0; v < V; ++v) acc[q][v] = fma(w, x[v], acc[q][v]);
            }
        }
    }
    if (is_long) {
#pragma unroll
        for (int q = 0; q < NOPS; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) red[(q * kBlock + threadIdx.x) * V + v] = acc[q][v];
        __syncthreads();
        if (grp != 0) return;
        for (int g = 1; g < GPB; ++g)
#pragma unroll
            for (int q = 0; q < NOPS; ++q)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[q][v] += red[(q * kBlock + g * G + lane) * V + v];
    }
    if (!active) return;
    const size_t off = (size_t)row * a.ld + col0;
    st_d(a.o0 + off, acc[0]);
    st_d(a.o1 + off, acc[1]);
    if (NOPS == 3) st_d(a.o2 + off, acc[NOPS - 1]);
}

template <typename TX, int G, int NOPS>
cudaError_t spmm_g(const SpmmArgs<TX>& a, cudaStream_t s) {
    constexpr int V = Vec<TX>::V, GPB = kBlock / G, TN = G * V;
    dim3 grid(a.n_long + (a.rows + GPB - 1) / GPB, (a.ncol + TN - 1) / TN);
    k_spmm64<TX, G, NOPS><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename TX, int NOPS>
cudaError_t spmm64(const Csr& m, const TX* s0, const TX* s1, const TX* s2, double* o0, double* o1, double* o2,
                   int ld, int ncol, cudaStream_t s) {
    if (m.rows == 0 || ncol == 0) return cudaSuccess;
    SpmmArgs<TX> a{m.rows, m.rp, m.ci, m.v64, m.long_rows, m.n_long, m.long_thr, s0, s1, s2, o0, o1, o2, ld, ncol};
    constexpr int V = Vec<TX>::V;
    const int vecs = (ncol + V - 1) / V;
    if (vecs <= 1) return spmm_g<TX, 1, NOPS>(a, s);
    if (vecs <= 2) return spmm_g<TX, 2, NOPS>(a, s);
    if (vecs <= 4) return spmm_g<TX, 4, NOPS>(a, s);
    if (vecs <= 8) return spmm_g<TX, 8, NOPS>(a, s);
    if (vecs <= 16) return spmm_g<TX, 16, NOPS>(a, s);
    return spmm_g<TX, 32, NOPS>(a, s);
}

// ---------------------------------------------------------------------------
// per-column partial sums over the rows (block 32 columns x kReduceRows rows)
// ---------------------------------------------------------------------------
template <int NS>
__device__ __forceinline__ void write_partials(double (&s)[NS], double* part, int stat0, int nb, int ld, int j,
                                               bool ok) {
    __shared__ double sh[kReduceRows][32];
    for (int q = 0; q < NS; ++q) {
        sh[threadIdx.y][threadIdx.x] = s[q];
        __syncthreads();
        if (threadIdx.y == 0) {
            double t = sh[0][threadIdx.x];
            for (int r = 1; r < kReduceRows; ++r) t += sh[r][threadIdx.x];
            if (ok) part[((size_t)(stat0 + q) * nb + blockIdx.x) * ld + j] = t;
        }
        __syncthreads();
    }
}

template <typename T>
struct ReduceArgs {
    int m, n, ld, ncol, nb_m, nb_n;
    const double *d_r, *d_c;
    const double *c, *xl, *xu, *l, *u;
    ColCheck col;
    const T *Xh, *DX, *G, *X0, *X, *Yh, *DY, *DYp, *Y0, *Y;
    const double *P0, *P1, *Q0, *Q1, *Q2;
    double* part;
    int restart_to_output;
    int robust_rc;  // 1: the stopping test takes the robust reduced cost
};

template <typename T>
__global__ void k_reduce_rows_m(const ReduceArgs<T> a) {
    const int j = blockIdx.y * 32 + threadIdx.x;
    const bool ok = j < a.ncol;
    double s[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q] = 0.0;
    if (ok) {
        for (int i = blockIdx.x * kReduceRows + threadIdx.y; i < a.m; i += gridDim.x * kReduceRows) {
            const size_t off = (size_t)i * a.ld + j;
            const double dr = a.d_r[i], l = a.l[i], u = a.u[i];
            const double ax = a.P0[off] / dr;               // A x, x = D_c x~
            const double pv = ax - proj_box(ax, l, u);
            s[0] += pv * pv;
            s[1] += ax * ax;
            const double yh = (double)a.Yh[off];
            s[2] += support(dr * yh, l, u);                 // phi_[l,u](y), y = D_r y~
            const double dy = (double)a.DY[off];
            s[3] += dy * dy;
            s[4] += dy * a.P1[off];                         // <dy~, A~ dx~>
            const double anchor = a.restart_to_output ? yh : (double)a.Y[off];
            const double dy0 = anchor - (double)a.Y0[off];
            s[5] += dy0 * dy0;
            s[6] += support(dr * (double)a.DYp[off], l, u); // phi(Pi_B(D_r dy~))
            const double adx = a.P1[off] / dr;              // A dx, dx = D_c dx~
            const double t = adx - proj_recession(adx, l, u);
            s[7] += t * t;
        }
    }
    write_partials<8>(s, a.part, S_PRES2, a.nb_m, a.ld, j, ok);
}

template <typename T>
__global__ void k_reduce_rows_n(const ReduceArgs<T> a) {
    const int j = blockIdx.y * 32 + threadIdx.x;
    const bool ok = j < a.ncol;
    double s[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) s[q] = 0.0;
    if (ok) {
        const int kind = a.col.kind[j], var = a.col.var[j];
        const double olo = a.col.lo[j], ohi = a.col.hi[j], oc = a.col.c[j];
        for (int i = blockIdx.x * kReduceRows + threadIdx.y; i < a.n; i += gridDim.x * kReduceRows) {
            const size_t off = (size_t)i * a.ld + j;
            const double dc = a.d_c[i];
            double cj = a.c[i], lo = a.xl[i], hi = a.xu[i];
            if (kind == 2) cj = var == i ? oc : 0.0;
            else if (kind == 1 && var == i) { lo = olo; hi = ohi; }
            const double xh = (double)a.Xh[off];
            const double x = proj_box(dc * xh, lo, hi);
            const double aty = a.Q0[off] / dc;              // A^T y
            const double q = cj + aty;
            const double r = proj_barrier(-q, lo, hi);      // reduced cost
            // the stopping test's reduced cost; the certificates keep Pi_B
            const double rs = a.robust_rc ? robust_rc(-q, x, lo, hi) : r;
            const double d = q + rs;
            s[0] += d * d;
            s[1] += cj * cj;
            s[2] += cj * x;
            s[3] += support(rs, lo, hi);
            const double dx = (double)a.DX[off];
            s[4] += dx * dx;
            const double anchor = a.restart_to_output ? xh : (double)a.X[off];
            const double dx0 = anchor - (double)a.X0[off];
            s[5] += dx0 * dx0;
            const double gk = (a.Q0[off] - a.Q2[off]) / dc; // A^T y^k = A^T y^ - A^T (y^ - y^k)
            const double rk = proj_barrier(-cj - gk, lo, hi);
            const double drr = proj_barrier(r - rk, lo, hi);
            s[6] += support(drr, lo, hi);
            const double t = a.Q1[off] / dc + drr;          // A^T dy + dr
            s[7] += t * t;
            const double dxo = dc * dx;
            s[8] += cj * dxo;
            const double t2 = dxo - proj_recession(dxo, lo, hi);
            s[9] += t2 * t2;
        }
    }
    write_partials<10>(s, a.part, S_DRES2, a.nb_n, a.ld, j, ok);
}

// colsum[s][j] = sum over the blocks' partials, in a fixed order.  The
// partials of statistic s start at s * kReduceBlocks * ld.
__global__ void k_colsum(const double* __restrict__ part, int nb_m, int nb_n, int ld, int ncol,
                         double* __restrict__ colsum) {
    __shared__ double sh[32][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int s = blockIdx.y;
    const int nb = s < S_DRES2 ? nb_m : nb_n;
    double acc = 0.0;
    if (j < ncol) {
        const double* p = part + (size_t)s * kReduceBlocks * ld;
        for (int b = threadIdx.y; b < nb; b += 32) acc += p[(size_t)b * ld + j];
    }
    sh[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    for (int w = 16; w > 0; w >>= 1) {
        if ((int)threadIdx.y < w) sh[threadIdx.y][threadIdx.x] += sh[threadIdx.y + w][threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.y == 0 && j < ncol) colsum[(size_t)s * ld + j] = sh[0][threadIdx.x];
}

// Halpern weights (k+1)/(k+2) and 1/(k+2) of Eq. mainiter for the
// iterations k0 .. k0+ce-1 of group g's next interval, computed once in FP64
// so that the iteration kernels do no division; thread `me` of `nth` writes
// every nth entry.
// Group g's Halpern weights (k+1)/(k+2), 1/(k+2) of Eq. mainiter for the
// interval that starts at inner index k0: entry e = 0 .. ce holds index
// k0 - 1 + e, so iteration t uses entry t + 1 and the primal step rebuilds
// its iterate with entry t; at k0 = 0 (a start or a restart) entry 0 is
// (0, 1): the iterate is the anchor.
__device__ __forceinline__ void write_halpern(double* hal64, float* hal32, dfloat* haldf, int g, int k0, int ce,
                                              int me, int nth) {
    for (int t = me; t <= ce; t += nth) {
        const double k = (double)k0 - 1.0 + t;
        const double ca = (k + 1.0) / (k + 2.0), cb = 1.0 / (k + 2.0);
        const size_t h = 2 * ((size_t)g * (ce + 1) + t);
        hal64[h] = ca;
        hal64[h + 1] = cb;
        hal32[h] = (float)ca;
        hal32[h + 1] = (float)cb;
        haldf[h] = dfloat(ca);
        haldf[h + 1] = dfloat(cb);
    }
}

template <typename T>
struct DecideArgs {
    const double* colsum;
    int ld, ncol;
    ColCheck col;
    ColParams<T> colp;
    double eta, mnorm_sign, beta_s, beta_n, beta_a, theta;
    int detect_inf, interval_len, stall_checks, check_every;
    ColRecord* rec;
    Control* ctl;     // gcap groups
    int gcap;
    double* hal64;
    float* hal32;
    dfloat* haldf;
    double* rscr;     // residual of each active LP at this check, by slot
    int* rtag;        // == this check's tag where rscr holds this check's value
    int* flags;       // [0]: some group restarted; [1]: check counter (the tag)
};

constexpr int kDecideThreads = 1024;

// Per-LP status from the summed statistics; then, for each restart group,
// the batch-averaged restart test (Sec. 5 "Restarts") over the group's
// active LPs, summed in slot order by a fixed tree so that a group's result
// does not depend on which columns its LPs occupy or what else runs beside
// it; on a restart, the primal-weight update of the group's active LPs.
template <typename T>
__global__ void __launch_bounds__(kDecideThreads) k_decide(const DecideArgs<T> a) {
    const size_t ld = (size_t)a.ld;
    __shared__ int sh_tag;
    for (int g = threadIdx.x; g < a.gcap; g += blockDim.x) a.ctl[g].stalled = 0;
    if (threadIdx.x == 0) {
        a.flags[0] = 0;
        sh_tag = a.flags[1] + 1;
        a.flags[1] = sh_tag;
    }
    __syncthreads();
    const int tag = sh_tag;
    for (int j = threadIdx.x; j < a.ncol; j += blockDim.x) {
        const int g = a.col.grp[j];
        const double tol = a.ctl[g].tol, eps_inf = a.ctl[g].eps_inf, tol_dual = a.ctl[g].tol_dual;
        double st[kNumStats];
        for (int s = 0; s < kNumStats; ++s) st[s] = a.colsum[s * ld + j];
        const double rel_p = sqrt(st[S_PRES2]) / (1.0 + sqrt(st[S_AX2]));
        const double rel_d = sqrt(st[S_DRES2]) / (1.0 + sqrt(st[S_C2]));
        const double dsum = st[S_PHR] + st[S_PHY];
        const double ctx = st[S_CTX];
        const double rel_g = isfinite(dsum) ? fabs(ctx + dsum) / (1.0 + fabs(ctx) + fabs(dsum)) : INFINITY;
        const double w = a.col.w[j];
        const double r2 = (w / a.eta) * st[S_DX2] + (1.0 / (a.eta * w)) * st[S_DY2] + 2.0 * a.mnorm_sign * st[S_CROSS];
        const double r = sqrt(r2 > 0.0 ? r2 : 0.0);
        int status = -1;
        if (isnan(ctx) || isnan(dsum) || isnan(rel_p) || isnan(rel_d) || isnan(rel_g) || !isfinite(r)) {
            status = LPB_NUMERICAL;
        } else if (rel_p <= tol && rel_d <= tol_dual && rel_g <= tol) {
            status = LPB_OPTIMAL;
        } else if (a.detect_inf) {
            const double ph = st[S_PHIDY] + st[S_PHIDR];
            const double cdx = st[S_CDX];
            if (ph < 0.0 && sqrt(st[S_RES2]) <= eps_inf * fabs(ph)) status = LPB_PRIMAL_INFEASIBLE;
            else if (cdx < 0.0 && sqrt(st[S_RX2]) <= eps_inf * fabs(cdx) &&
                     sqrt(st[S_RA2]) <= eps_inf * fabs(cdx))
                status = LPB_DUAL_INFEASIBLE;
        }
        ColRecord rc;
        rc.status = status;
        rc.pad = 0;
        rc.r = r;
        rc.obj = ctx;
        rc.dual_obj = -dsum;
        rc.rel_primal = rel_p;
        rc.rel_dual = rel_d;
        rc.rel_gap = rel_g;
        // the dual bound shifted by Delta = tol (1 + |c^T x| + |phi + phi|) (Sec. 6, OBBT)
        rc.safe = -dsum - tol * (1.0 + fabs(ctx) + fabs(dsum));
        a.rec[j] = rc;
        if (status < 0) {
            const int slot = a.col.slot[j];
            a.rscr[slot] = r;
            a.rtag[slot] = tag;
            if (a.stall_checks > 0) {
                // an LP stalls when its KKT error has not halved for stall_checks checks
                const double err = fmax(rel_p, fmax(rel_d, rel_g));
                if (err < 0.5 * a.col.best[j]) {
                    a.col.best[j] = err;
                    a.col.stall[j] = 0;
                } else if (++a.col.stall[j] >= a.stall_checks) {
                    a.ctl[g].stalled = 1;
                }
            }
        }
    }
    __syncthreads();
    // one warp per group: the averaged residual and the restart test
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int g = warp; g < a.gcap; g += blockDim.x >> 5) {
        Control* c = a.ctl + g;
        if (!c->active) continue;
        double sum = 0.0;
        int cnt = 0;
        for (int q = lane; q < c->nslots; q += 32) {
            const int slot = c->slot0 + q;
            if (a.rtag[slot] == tag) {
                sum += a.rscr[slot];
                ++cnt;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            sum += __shfl_down_sync(kFull, sum, o);
            cnt += __shfl_down_sync(kFull, cnt, o);
        }
        int k_next = 0;
        if (lane == 0) {
            const int L = a.interval_len;
            const bool final_check = c->K + L >= c->max_iter;
            int restart = 0;
            const double rt = cnt > 0 ? sum / cnt : 0.0;
            if (cnt > 0 && !final_check) {
                if (c->r0 < 0.0) {
                    c->r0 = rt;
                    c->r_prev = rt;
                }
                const long long k_eval = (long long)c->k + L - 1;
                const long long k_eval_global = (long long)c->K + L - 1;
                restart = (rt <= a.beta_s * c->r0) || (rt <= a.beta_n * c->r0 && rt > c->r_prev) ||
                          ((double)k_eval > a.beta_a * (double)k_eval_global);
                if (restart) {
                    c->k = 0;
                    c->r0 = rt;
                    c->r_prev = rt;
                    c->restarts += 1;
                    atomicOr(a.flags, 1);
                } else {
                    c->k += L;
                    c->r_prev = rt;
                }
            }
            c->K += L;
            c->restart = restart;
            c->r_avg = rt;
            k_next = c->k;
        }
        k_next = __shfl_sync(kFull, k_next, 0);
        write_halpern(a.hal64, a.hal32, a.haldf, g, k_next, a.check_every, lane, 32);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < a.ncol; j += blockDim.x) {
        if (a.rec[j].status >= 0 || !a.ctl[a.col.grp[j]].restart) continue;
        const double ddx = a.colsum[S_DX02 * ld + j], ddy = a.colsum[S_DY02 * ld + j];
        const double d = sqrt(ddy) / sqrt(ddx);   // ||y^{n+1,0} - y^{n,0}|| / ||x^{n+1,0} - x^{n,0}||
        if (ddx > 0.0 && ddy > 0.0 && isfinite(d) && d > 0.0) {
            const double w = exp(a.theta * log(d) + (1.0 - a.theta) * log(a.col.w[j]));
            a.col.w[j] = w;
            a.colp.tau[j] = (T)(a.eta / w);
            a.colp.sigma[j] = (T)(a.eta * w);
        }
    }
}

// On a restart of a column's group: anchor and iterate <- T(z) at the check
// (or the anchor <- the Halpern iterate for restart_to_output = 0).  The
// dual side keeps its iterate Z; the primal side keeps only the reflected
// point Zbar, from which the next step rebuilds the iterate (with weights
// 0 and 1 after a restart), and sets it to the new anchor as well.
template <typename T>
__global__ void k_restart_copy(T* __restrict__ Z, T* __restrict__ Zbar, T* __restrict__ Z0,
                               const T* __restrict__ Zh, int rows, int ld, int ncol, int to_output,
                               const int* __restrict__ grp, const Control* __restrict__ ctl,
                               const int* __restrict__ flags) {
    if (!flags[0]) return;
    const size_t total = (size_t)rows * ld;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(p % ld);
        if (j >= ncol || !ctl[grp[j]].restart) continue;
        const T v = to_output ? Zh[p] : Z[p];
        if (Z && to_output) Z[p] = v;
        if (Zbar) Zbar[p] = v;
        Z0[p] = v;
    }
}

// The primal Halpern iterate after an interval of L iterations,
// X = (k+1)/(k+2) Xbar + X^0/(k+2) with the weights of the interval's last
// iteration (entry L of the column's group), for the checks of
// restart_to_output = 0, which read the iterate itself.
template <typename T>
__global__ void k_halpern_iterate(T* __restrict__ X, const T* __restrict__ Xbar, const T* __restrict__ X0,
                                  const T* __restrict__ hal, const int* __restrict__ grp, int rows, int ld, int ncol,
                                  int ce, int L) {
    const size_t total = (size_t)rows * ld;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(p % ld);
        if (j >= ncol) continue;
        const size_t h = 2 * ((size_t)grp[j] * (ce + 1) + L);
        X[p] = hal[h] * Xbar[p] + hal[h + 1] * X0[p];
    }
}

// ---------------------------------------------------------------------------
// batch set-up, extraction, compaction
// ---------------------------------------------------------------------------
template <typename T>
struct InitArgs {
    int m, n, ld;
    int c0, count;                       // admitted columns [c0, c0 + count)
    int group, slot0;                    // their restart group and first residual slot
    const lpb_lp_spec* specs;            // count records
    const double *d_r, *d_c, *xl, *xu;   // original box
    const T *xls, *xus;                  // scaled box, iterate precision
    double eta, c_norm_base, b_norm;
    ColParams<T> colp;
    ColCheck colc;
    ColRecord* rec;
    Control* ctl;
};

// A new restart group g owning residual slots [slot0, slot0 + nslots); runs
// before k_init_columns, whose threads may raise ctl[g].error.
__global__ void k_admit_group(Control* ctl, int g, int slot0, int nslots, double tol, double eps_inf,
                              double tol_dual, long long max_iter, double* hal64, float* hal32, dfloat* haldf,
                              int ce) {
    if (threadIdx.x == 0) {
        Control c{};
        c.k = 0;
        c.restart = 0;
        c.error = 0;
        c.stalled = 0;
        c.r0 = -1.0;
        c.r_prev = -1.0;
        c.r_avg = 0.0;
        c.restarts = 0;
        c.K = 0;
        c.max_iter = max_iter;
        c.tol = tol;
        c.eps_inf = eps_inf;
        c.tol_dual = tol_dual;
        c.slot0 = slot0;
        c.nslots = nslots;
        c.active = 1;
        c.pad = 0;
        ctl[g] = c;
    }
    write_halpern(hal64, hal32, haldf, g, 0, ce, threadIdx.x, blockDim.x);
}

// Group g now lives at ctl[g] of another lane (copied there by the host):
// its slots move to slot0 and its Halpern table is written for its k.
__global__ void k_group_moved(Control* ctl, int g, int slot0, double* hal64, float* hal32, dfloat* haldf, int ce) {
    const int k = ctl[g].k;
    __syncthreads();
    if (threadIdx.x == 0) ctl[g].slot0 = slot0;
    write_halpern(hal64, hal32, haldf, g, k, ce, threadIdx.x, blockDim.x);
}

template <typename T>
__global__ void k_init_columns(const InitArgs<T> a) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= a.count) return;
    const int j = a.c0 + q;
    Control* ctl = a.ctl + a.group;
    int kind = 0, var = -1;
    double olo = 0.0, ohi = 0.0, oc = 0.0;
    T slo = T(0), shi = T(0), sc = T(0);
    double cn = a.c_norm_base;
    int status = -1;
    const lpb_lp_spec sp = a.specs[q];
    kind = sp.kind;
    var = sp.var;
    if (kind < 0 || kind > 2) {
        atomicMax(&ctl->error, (int)LPB_ERR_INVALID_ARG);
        kind = 0;
    }
    if (kind != 0 && (var < 0 || var >= a.n)) {
        atomicMax(&ctl->error, (int)LPB_ERR_BAD_INDEX);
        kind = 0;
    }
    if (kind == 0) var = -1;
    if (kind == 1) {
        olo = sp.lo > a.xl[var] ? sp.lo : a.xl[var];
        ohi = sp.hi < a.xu[var] ? sp.hi : a.xu[var];
        if (isnan(sp.lo) || isnan(sp.hi)) atomicMax(&ctl->error, (int)LPB_ERR_INVALID_ARG);
        if (olo > ohi) status = LPB_PRIMAL_INFEASIBLE;
        slo = (T)(olo / a.d_c[var]);
        shi = (T)(ohi / a.d_c[var]);
    } else if (kind == 2) {
        if (!isfinite(sp.sign)) atomicMax(&ctl->error, (int)LPB_ERR_INVALID_ARG);
        oc = sp.sign;
        sc = (T)(a.d_c[var] * sp.sign);
        cn = fabs(a.d_c[var] * sp.sign);
    }
    double w = 1.0;
    const double w0 = cn / a.b_norm;
    if (cn > 0.0 && a.b_norm > 0.0 && isfinite(w0)) w = w0;
    a.colp.kind[j] = kind;
    a.colp.var[j] = var;
    a.colp.grp[j] = a.group;
    a.colp.lo[j] = slo;
    a.colp.hi[j] = shi;
    a.colp.c[j] = sc;
    a.colp.tau[j] = (T)(a.eta / w);
    a.colp.sigma[j] = (T)(a.eta * w);
    a.colc.kind[j] = kind;
    a.colc.var[j] = var;
    a.colc.lo[j] = olo;
    a.colc.hi[j] = ohi;
    a.colc.c[j] = oc;
    a.colc.w[j] = w;
    a.colc.slot[j] = a.slot0 + q;
    a.colc.best[j] = INFINITY;
    a.colc.stall[j] = 0;
    ColRecord rc;
    rc.status = status;
    rc.pad = 0;
    rc.r = 0.0;
    rc.obj = rc.dual_obj = rc.rel_primal = rc.rel_dual = rc.rel_gap = rc.safe = NAN;
    a.rec[j] = rc;
}

// z0 = (Pi_box(warm_x / D_c), warm_y / D_r), or (Pi_box(0), 0), for the
// admitted columns; LP q's warm start is warm_x + q * wsx (n values) and
// warm_y + q * wsy (m values): column-major blocks, or one vector for every
// LP with stride 0
// (the primal side stores the reflected point Xbar, from which the first
// step rebuilds the iterate with weights 0 and 1: it starts equal to X0)
template <typename T>
__global__ void k_init_iterates(const InitArgs<T> a, T* Xbar, T* X0, T* Y, T* Y0, const double* warm_x,
                                const double* warm_y, long long wsx, long long wsy) {
    const size_t nx = (size_t)a.n * a.count, ny = (size_t)a.m * a.count;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < nx + ny; p += (size_t)gridDim.x * blockDim.x) {
        if (p < nx) {
            const int i = (int)(p / a.count), q = (int)(p % a.count);
            const int j = a.c0 + q;
            T lo = a.xls[i], hi = a.xus[i];
            const int kind = a.colp.kind[j];
            if (kind == 1 && a.colp.var[j] == i) { lo = a.colp.lo[j]; hi = a.colp.hi[j]; }
            const T w = warm_x ? (T)(warm_x[q * wsx + i] / a.d_c[i]) : T(0);
            T t = w < hi ? w : hi;
            const T v = t > lo ? t : lo;
            const size_t e = (size_t)i * a.ld + j;
            Xbar[e] = v;
            X0[e] = v;
        } else {
            const size_t r = p - nx;
            const int i = (int)(r / a.count), q = (int)(r % a.count);
            const T v = warm_y ? (T)(warm_y[q * wsy + i] / a.d_r[i]) : T(0);
            const size_t e = (size_t)i * a.ld + a.c0 + q;
            Y[e] = v;
            Y0[e] = v;
        }
    }
}

// finished column cols[f] -> x at outp[f] (n) and y at outp[count + f] (m),
// in the original space
template <typename T>
__global__ void k_extract(int n, int m, int ld, const int* __restrict__ cols, double* const* __restrict__ outp,
                          int count, const double* __restrict__ d_r, const double* __restrict__ d_c,
                          const double* __restrict__ xl, const double* __restrict__ xu, ColCheck colc,
                          const T* __restrict__ Xh, const T* __restrict__ Yh) {
    const int f = blockIdx.y;
    if (f >= count) return;
    const int j = cols[f];
    double* x_out = outp[f];
    double* y_out = outp[count + f];
    const int kind = colc.kind[j], var = colc.var[j];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < (n > m ? n : m); i += gridDim.x * blockDim.x) {
        if (i < n && x_out) {
            double lo = xl[i], hi = xu[i];
            if (kind == 1 && var == i) { lo = colc.lo[j]; hi = colc.hi[j]; }
            x_out[i] = proj_box(d_c[i] * (double)Xh[(size_t)i * ld + j], lo, hi);
        }
        if (i < m && y_out) y_out[i] = d_r[i] * (double)Yh[(size_t)i * ld + j];
    }
}

// moves column src[p] -> dst[p] in every row of the state blocks (the
// primal reflected point Xbar and anchor X0, the dual iterate and anchor)
template <typename T>
__global__ void k_compact_rows(T* X, T* X0, T* Y, T* Y0, int n, int m, int ld, const int* __restrict__ src,
                               const int* __restrict__ dst, int count) {
    const size_t total = (size_t)(n + m) * count;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int mv = (int)(p % count);
        const int row = (int)(p / count);
        const int s = src[mv], d = dst[mv];
        if (row < n) {
            const size_t r = (size_t)row * ld;
            X[r + d] = X[r + s];
            X0[r + d] = X0[r + s];
        } else {
            const size_t r = (size_t)(row - n) * ld;
            Y[r + d] = Y[r + s];
            Y0[r + d] = Y0[r + s];
        }
    }
}

template <typename T>
__global__ void k_compact_cols(ColParams<T> cp, ColCheck cc, const int* __restrict__ src, const int* __restrict__ dst,
                               int count) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const int s = src[p], d = dst[p];
    cp.kind[d] = cp.kind[s];
    cp.var[d] = cp.var[s];
    cp.grp[d] = cp.grp[s];
    cp.lo[d] = cp.lo[s];
    cp.hi[d] = cp.hi[s];
    cp.c[d] = cp.c[s];
    cp.tau[d] = cp.tau[s];
    cp.sigma[d] = cp.sigma[s];
    cc.lo[d] = cc.lo[s];
    cc.hi[d] = cc.hi[s];
    cc.c[d] = cc.c[s];
    cc.w[d] = cc.w[s];
    cc.slot[d] = cc.slot[s];
    cc.best[d] = cc.best[s];
    cc.stall[d] = cc.stall[s];
}

inline int blocks_for(size_t work, int threads, int cap = 8192) {
    size_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------------------
// double-float checks for FP32 and dfloat iterates.  The FP64 versions above
// run for FP64 iterates; these give FP64-level accuracy on the FP32 pipe.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ldg_it(const float* p, float (&r)[4]) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = u.x; r[1] = u.y; r[2] = u.z; r[3] = u.w;
}
__device__ __forceinline__ void ldg_it(const dfloat* p, dfloat (&r)[2]) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = dfloat(u.x, u.y); r[1] = dfloat(u.z, u.w);
}
// an iterate value as FP32 (norms) and as df (terms that cancel)
__device__ __forceinline__ float it_f(float v) { return v; }
__device__ __forceinline__ float it_f(dfloat v) { return v.hi + v.lo; }
__device__ __forceinline__ df it_mul(df a, float v) { return df_mulf(a, v); }
__device__ __forceinline__ df it_mul(df a, dfloat v) { return df_mul(a, df_of(v)); }
// a - b rounded to FP32 (exact leading parts by Sterbenz when close)
__device__ __forceinline__ float it_diff(float a, float b) { return a - b; }
__device__ __forceinline__ float it_diff(dfloat a, dfloat b) { return (a.hi - b.hi) + (a.lo - b.lo); }

template <typename TI>
struct SpmmDfArgs {
    int rows;
    const int* rp;
    const int* ci;
    const float* vhi;   // A~ in double-float: vhi + vlo
    const float* vlo;
    const int* long_rows;
    int n_long, long_thr;
    const TI* s0;
    const TI* s1;
    const TI* s2;
    df* o0;
    df* o1;
    df* o2;
    int ld, ncol;
};

// o_q = A~ s_q for NOPS operands, each product a_e * x accumulated exactly
template <typename TI, int G, int NOPS>
__global__ void __launch_bounds__(kBlock) k_spmm_df(const SpmmDfArgs<TI> a) {
    constexpr int V = Vec<TI>::V, GPB = kBlock / G, TN = G * V;
    __shared__ df red[NOPS * kBlock * V];
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int col0 = blockIdx.y * TN + lane * V;
    const bool active = col0 < a.ncol;
    const bool is_long = (int)blockIdx.x < a.n_long;
    int row, slot = 0, nslot = 1;
    if (is_long) {
        row = a.long_rows[blockIdx.x];
        slot = grp;
        nslot = GPB;
    } else {
        row = ((int)blockIdx.x - a.n_long) * GPB + grp;
        if (row >= a.rows) return;
        if (a.rp[row + 1] - a.rp[row] > a.long_thr) return;
    }
    df acc[NOPS][V];
#pragma unroll
    for (int q = 0; q < NOPS; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[q][v] = df_zero();
    const TI* src[3] = {a.s0, a.s1, a.s2};
    if (active) {
        const int end = a.rp[row + 1];
        int e = a.rp[row] + slot;
        // four of the slot's entries per round: their gathers are issued
        // together (loads in flight), the sums still taken in entry order
        for (; e + 3 * nslot < end; e += 4 * nslot) {
            int c[4];
            df w[4];
            TI x[4][NOPS][V];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                c[k] = a.ci[e + k * nslot];
                w[k] = df{a.vhi[e + k * nslot], a.vlo[e + k * nslot]};
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int q = 0; q < NOPS; ++q) ldg_it(src[q] + (size_t)c[k] * a.ld + col0, x[k][q]);
#pragma unroll
            for (int k = 0; k < 4; ++k)
#pragma unroll
                for (int q = 0; q < NOPS; ++q)
#pragma unroll
                    for (int v = 0; v < V; ++v) df_fma_acc(acc[q][v], w[k], x[k][q][v]);
        }
        for (; e < end; e += nslot) {
            const int c = a.ci[e];
            const df w = df{a.vhi[e], a.vlo[e]};
#pragma unroll
            for (int q = 0; q < NOPS; ++q) {
                TI x[V];
                ldg_it(src[q] + (size_t)c * a.ld + col0, x);
#pragma unroll
                for (int v = 0; v < V; ++v) df_fma_acc(acc[q][v], w, x[v]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NOPS; ++q)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[q][v] = quick_two_sum(acc[q][v].hi, acc[q][v].lo);
    if (is_long) {
#pragma unroll
        for (int q = 0; q < NOPS; ++q)
#pragma unroll
            for (int v = 0; v < V; ++v) red[(q * kBlock + threadIdx.x) * V + v] = acc[q][v];
        __syncthreads();
        if (grp != 0) return;
        for (int g = 1; g < GPB; ++g)
#pragma unroll
            for (int q = 0; q < NOPS; ++q)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[q][v] = df_add(acc[q][v], red[(q * kBlock + g * G + lane) * V + v]);
    }
    if (!active) return;
    const size_t off = (size_t)row * a.ld + col0;
    df* out[3] = {a.o0, a.o1, a.o2};
#pragma unroll
    for (int q = 0; q < NOPS; ++q) {
        float4* p = reinterpret_cast<float4*>(out[q] + off);
#pragma unroll
        for (int v = 0; v < V; v += 2)
            p[v / 2] = make_float4(acc[q][v].hi, acc[q][v].lo, acc[q][v + 1].hi, acc[q][v + 1].lo);
    }
}

template <typename TI, int NOPS>
cudaError_t spmm_df(const Csr& m, const TI* s0, const TI* s1, const TI* s2, df* o0, df* o1, df* o2, int ld,
                    int ncol, cudaStream_t s) {
    if (m.rows == 0 || ncol == 0) return cudaSuccess;
    constexpr int V = Vec<TI>::V;
    SpmmDfArgs<TI> a{m.rows, m.rp,   m.ci, m.v32, m.v32lo, m.long_rows, m.n_long,
                     m.long_thr, s0, s1, s2, o0,   o1,    o2,          ld,       ncol};
    const int vecs = (ncol + V - 1) / V;
    const int G = vecs <= 1 ? 1 : vecs <= 2 ? 2 : vecs <= 4 ? 4 : vecs <= 8 ? 8 : vecs <= 16 ? 16 : 32;
    const int gpb = kBlock / G, tn = G * V;
    dim3 grid(a.n_long + (a.rows + gpb - 1) / gpb, (ncol + tn - 1) / tn);
    switch (G) {
        case 1: k_spmm_df<TI, 1, NOPS><<<grid, kBlock, 0, s>>>(a); break;
        case 2: k_spmm_df<TI, 2, NOPS><<<grid, kBlock, 0, s>>>(a); break;
        case 4: k_spmm_df<TI, 4, NOPS><<<grid, kBlock, 0, s>>>(a); break;
        case 8: k_spmm_df<TI, 8, NOPS><<<grid, kBlock, 0, s>>>(a); break;
        case 16: k_spmm_df<TI, 16, NOPS><<<grid, kBlock, 0, s>>>(a); break;
        default: k_spmm_df<TI, 32, NOPS><<<grid, kBlock, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

__device__ __forceinline__ float proj_recession_f(float v, float a, float b) {
    const bool li = isinf(a), hi = isinf(b);
    if (li && hi) return v;
    if (hi) return v > 0.0f ? v : 0.0f;
    if (li) return v < 0.0f ? v : 0.0f;
    return 0.0f;
}

__device__ __forceinline__ df df_from(double v) {
    const float hi = (float)v;
    return df{hi, isfinite(v) && isfinite(hi) ? (float)(v - (double)hi) : 0.0f};
}

template <typename TI>
struct ReduceDfArgs {
    int m, n, ld, ncol;
    const df *dr, *dc, *idr, *idc, *c, *xl, *xu, *l, *u;
    ColCheck col;
    const TI *Xh, *DX, *X0, *X, *Yh, *DY, *DYp, *Y0, *Y;
    const df *P0, *P1, *Q0, *Q1, *Q2;
    double* part;
    int restart_to_output;
    int robust_rc;  // 1: the stopping test takes the robust reduced cost
};

// m-side statistics (the same quantities as k_reduce_rows_m); the terms that
// cancel (A x against its bounds, phi sums) in double-float, norms in FP32
template <typename TI>
__global__ void k_reduce_m_df(const ReduceDfArgs<TI> a) {
    const int j = blockIdx.y * 32 + threadIdx.x;
    const bool ok = j < a.ncol;
    float f_pres2 = 0.f, f_ax2 = 0.f, f_dy2 = 0.f, f_cross = 0.f, f_dy02 = 0.f, f_ra2 = 0.f;
    df d_phy = df_zero(), d_phidy = df_zero();
    if (ok) {
        for (int i = blockIdx.x * kReduceRows + threadIdx.y; i < a.m; i += gridDim.x * kReduceRows) {
            const size_t off = (size_t)i * a.ld + j;
            const df dr = a.dr[i], idr = a.idr[i], l = a.l[i], u = a.u[i];
            const df ax = df_mul(a.P0[off], idr);                    // A x, x = D_c x~
            const float pv = df_f(df_sub(ax, df_clamp(ax, l, u)));
            f_pres2 += pv * pv;
            f_ax2 += ax.hi * ax.hi;
            const TI yh = a.Yh[off];
            df_acc(d_phy, df_support(it_mul(dr, yh), l, u));          // phi_[l,u](y), y = D_r y~
            const float dy = it_f(a.DY[off]);
            f_dy2 += dy * dy;
            const float p1 = df_f(a.P1[off]);
            f_cross += dy * p1;                                      // <dy~, A~ dx~>
            const float dy0 = it_diff(a.restart_to_output ? yh : a.Y[off], a.Y0[off]);
            f_dy02 += dy0 * dy0;
            df_acc(d_phidy, df_support(it_mul(dr, a.DYp[off]), l, u));
            const float adx = df_f(df_mulf(idr, p1));                // A dx, dx = D_c dx~
            const float t = adx - proj_recession_f(adx, l.hi, u.hi);
            f_ra2 += t * t;
        }
    }
    double s[8] = {f_pres2, f_ax2, df_d(d_phy), f_dy2, f_cross, f_dy02, df_d(d_phidy), f_ra2};
    write_partials<8>(s, a.part, S_PRES2, kReduceBlocks, a.ld, j, ok);
}

template <typename TI>
__global__ void k_reduce_n_df(const ReduceDfArgs<TI> a) {
    const int j = blockIdx.y * 32 + threadIdx.x;
    const bool ok = j < a.ncol;
    float f_dres2 = 0.f, f_c2 = 0.f, f_dx2 = 0.f, f_dx02 = 0.f, f_res2 = 0.f, f_rx2 = 0.f;
    df d_ctx = df_zero(), d_phr = df_zero(), d_phidr = df_zero(), d_cdx = df_zero();
    if (ok) {
        const int kind = a.col.kind[j], var = a.col.var[j];
        const df olo = df_from(a.col.lo[j]), ohi = df_from(a.col.hi[j]), oc = df_from(a.col.c[j]);
        for (int i = blockIdx.x * kReduceRows + threadIdx.y; i < a.n; i += gridDim.x * kReduceRows) {
            const size_t off = (size_t)i * a.ld + j;
            const df dc = a.dc[i], idc = a.idc[i];
            df cj = a.c[i], lo = a.xl[i], hi = a.xu[i];
            if (kind == 2) cj = var == i ? oc : df_zero();
            else if (kind == 1 && var == i) { lo = olo; hi = ohi; }
            const TI xh = a.Xh[off];
            const df x = df_clamp(it_mul(dc, xh), lo, hi);
            const df q = df_add(cj, df_mul(a.Q0[off], idc));         // c + A^T y
            const df r = df_barrier(df_neg(q), lo, hi);              // reduced cost
            // the stopping test's reduced cost; the certificates keep Pi_B
            const df rs = a.robust_rc ? df_robust_rc(df_neg(q), x, lo, hi) : r;
            const float d = df_f(df_add(q, rs));
            f_dres2 += d * d;
            f_c2 += cj.hi * cj.hi;
            df_acc(d_ctx, df_mul(cj, x));
            df_acc(d_phr, df_support(rs, lo, hi));
            const TI dx = a.DX[off];
            const float dxs = it_f(dx);
            f_dx2 += dxs * dxs;
            const float dx0 = it_diff(a.restart_to_output ? xh : a.X[off], a.X0[off]);
            f_dx02 += dx0 * dx0;
            // A^T y^k = A^T y^ - A^T (y^ - y^k)
            const df gk = df_mul(df_sub(a.Q0[off], a.Q2[off]), idc);
            const df rk = df_barrier(df_neg(df_add(cj, gk)), lo, hi);
            const df drr = df_barrier(df_sub(r, rk), lo, hi);
            df_acc(d_phidr, df_support(drr, lo, hi));
            const float t = df_f(df_add(df_mul(a.Q1[off], idc), drr)); // A^T dy + dr
            f_res2 += t * t;
            const df dxo = it_mul(dc, dx);
            df_acc(d_cdx, df_mul(cj, dxo));
            const float dxf = df_f(dxo);
            const float t2 = dxf - proj_recession_f(dxf, lo.hi, hi.hi);
            f_rx2 += t2 * t2;
        }
    }
    double s[10] = {f_dres2, f_c2, df_d(d_ctx), df_d(d_phr), f_dx2, f_dx02, df_d(d_phidr), f_res2, df_d(d_cdx), f_rx2};
    write_partials<10>(s, a.part, S_DRES2, kReduceBlocks, a.ld, j, ok);
}

// The n-side check in one pass, for a transpose without long rows: thread
// (x, y) of a block takes column j of its 32-column tile and rows y, y + 8,
// ... of the block's row set (the same rows and order as k_reduce_n_df);
// for each row it forms c + A^T y^, A^T Pi_B(dy) and A^T dy from the row's
// entries in double-float (the warp shares the row's entries, each thread
// gathers its column) and folds them straight into the per-column
// statistics, so the three n x N products never go to memory.
// (four resident blocks per SM: the batched gathers would otherwise take the
// registers of a fourth block)
template <typename TI>
__global__ void __launch_bounds__(32 * kReduceRows, 4)
    k_check_n_df(const ReduceDfArgs<TI> a, const int* __restrict__ rp, const int* __restrict__ ci,
                 const float* __restrict__ vhi, const float* __restrict__ vlo) {
    const int j = blockIdx.y * 32 + threadIdx.x;
    const bool ok = j < a.ncol;
    const int jj = ok ? j : blockIdx.y * 32;  // lanes past the last LP read a valid column
    float f_dres2 = 0.f, f_c2 = 0.f, f_dx2 = 0.f, f_dx02 = 0.f, f_res2 = 0.f, f_rx2 = 0.f;
    df d_ctx = df_zero(), d_phr = df_zero(), d_phidr = df_zero(), d_cdx = df_zero();
    const int kind = a.col.kind[jj], var = a.col.var[jj];
    const df olo = df_from(a.col.lo[jj]), ohi = df_from(a.col.hi[jj]), oc = df_from(a.col.c[jj]);
    for (int i = blockIdx.x * kReduceRows + threadIdx.y; i < a.n; i += gridDim.x * kReduceRows) {
        // the row's own operands, issued before its gathers so that their
        // round trip overlaps the gathers' rather than following them
        const size_t off = (size_t)i * a.ld + jj;
        const TI xh = a.Xh[off];
        const TI dx = a.DX[off];
        const TI x0 = a.X0[off];
        // A~^T [y^, Pi_B(dy), dy] for row i, column j: the gathers of four
        // entries are issued together (loads in flight), the sums still taken
        // in entry order
        df q0 = df_zero(), q1 = df_zero(), q2 = df_zero();
        const int end = rp[i + 1];
        int e = rp[i];
        for (; e + 4 <= end; e += 4) {
            size_t src[4];
            df w[4];
            TI g0[4], g1[4], g2[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                src[k] = (size_t)ci[e + k] * a.ld + jj;
                w[k] = df{vhi[e + k], vlo[e + k]};
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                g0[k] = a.Yh[src[k]];
                g1[k] = a.DYp[src[k]];
                g2[k] = a.DY[src[k]];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                df_fma_acc(q0, w[k], g0[k]);
                df_fma_acc(q1, w[k], g1[k]);
                df_fma_acc(q2, w[k], g2[k]);
            }
        }
        for (; e < end; ++e) {
            const size_t src = (size_t)ci[e] * a.ld + jj;
            const df w = df{vhi[e], vlo[e]};
            df_fma_acc(q0, w, a.Yh[src]);
            df_fma_acc(q1, w, a.DYp[src]);
            df_fma_acc(q2, w, a.DY[src]);
        }
        q0 = quick_two_sum(q0.hi, q0.lo);
        q1 = quick_two_sum(q1.hi, q1.lo);
        q2 = quick_two_sum(q2.hi, q2.lo);
        const df dc = a.dc[i], idc = a.idc[i];
        df cj = a.c[i], lo = a.xl[i], hi = a.xu[i];
        if (kind == 2) cj = var == i ? oc : df_zero();
        else if (kind == 1 && var == i) { lo = olo; hi = ohi; }
        const df x = df_clamp(it_mul(dc, xh), lo, hi);
        const df q = df_add(cj, df_mul(q0, idc));                    // c + A^T y
        const df r = df_barrier(df_neg(q), lo, hi);                  // reduced cost
        // the stopping test's reduced cost; the certificates keep Pi_B
        const df rs = a.robust_rc ? df_robust_rc(df_neg(q), x, lo, hi) : r;
        const float d = df_f(df_add(q, rs));
        f_dres2 += d * d;
        f_c2 += cj.hi * cj.hi;
        df_acc(d_ctx, df_mul(cj, x));
        df_acc(d_phr, df_support(rs, lo, hi));
        const float dxs = it_f(dx);
        f_dx2 += dxs * dxs;
        const float dx0 = it_diff(a.restart_to_output ? xh : a.X[off], x0);
        f_dx02 += dx0 * dx0;
        // A^T y^k = A^T y^ - A^T (y^ - y^k)
        const df gk = df_mul(df_sub(q0, q2), idc);
        const df rk = df_barrier(df_neg(df_add(cj, gk)), lo, hi);
        const df drr = df_barrier(df_sub(r, rk), lo, hi);
        df_acc(d_phidr, df_support(drr, lo, hi));
        const float t = df_f(df_add(df_mul(q1, idc), drr));          // A^T dy + dr
        f_res2 += t * t;
        const df dxo = it_mul(dc, dx);
        df_acc(d_cdx, df_mul(cj, dxo));
        const float dxf = df_f(dxo);
        const float t2 = dxf - proj_recession_f(dxf, lo.hi, hi.hi);
        f_rx2 += t2 * t2;
    }
    double s[10] = {f_dres2, f_c2, df_d(d_ctx), df_d(d_phr), f_dx2, f_dx02, df_d(d_phidr), f_res2, df_d(d_cdx), f_rx2};
    write_partials<10>(s, a.part, S_DRES2, kReduceBlocks, a.ld, j, ok);
}

}  // namespace

template <typename T>
cudaError_t launch_check(const CheckData& d, const IterBufs<T>& b, int ld, int ncol, int interval_len,
                         double* P, double* Q, double* partials, double* colsum, ColRecord* rec, ColParams<T> colp,
                         cudaStream_t s, cudaEvent_t* ev) {
    cudaError_t e;
    const int m = d.m, n = d.n;
    double* P0 = P;
    double* P1 = P + (size_t)(m > 0 ? m : 1) * ld;
    double* Q0 = Q;
    double* Q1 = Q + (size_t)n * ld;
    double* Q2 = Q + 2 * (size_t)n * ld;
    constexpr bool kDf = !std::is_same<T, double>::value;  // FP32 or dfloat iterates
    if (ev && (e = cudaEventRecord(ev[0], s)) != cudaSuccess) return e;
    if (!d.restart_to_output) {
        // the checks of the literal restart reading read the Halpern iterate
        const T* hal = std::is_same<T, double>::value ? (const T*)d.hal64
                       : std::is_same<T, float>::value ? (const T*)d.hal32 : (const T*)d.haldf;
        k_halpern_iterate<T><<<blocks_for((size_t)n * ld, 256), 256, 0, s>>>(b.X, b.Xbar, b.X0, hal, d.col.grp, n, ld,
                                                                             ncol, d.check_every, interval_len);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // A~ [x^, x^ - x] and A~^T [y^, Pi_B(y^ - y), y^ - y]: in double-float for
    // FP32 iterates, in FP64 for FP64 iterates (P and Q hold either)
    if constexpr (kDf) {
        if ((e = spmm_df<T, 2>(d.A, b.Xh, b.DX, nullptr, (df*)P0, (df*)P1, nullptr, ld, ncol, s)) != cudaSuccess)
            return e;
        // without long rows in A~^T the n-side products are formed inside the
        // n-side reduction (k_check_n_df)
        if (d.At.n_long > 0 &&
            (e = spmm_df<T, 3>(d.At, b.Yh, b.DYp, b.DY, (df*)Q0, (df*)Q1, (df*)Q2, ld, ncol, s)) != cudaSuccess)
            return e;
    } else {
        if ((e = spmm64<T, 2>(d.A, b.Xh, b.DX, nullptr, P0, P1, nullptr, ld, ncol, s)) != cudaSuccess) return e;
        if ((e = spmm64<T, 3>(d.At, b.Yh, b.DYp, b.DY, Q0, Q1, Q2, ld, ncol, s)) != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[1], s)) != cudaSuccess) return e;

    const int tiles = (ncol + 31) / 32;
    const int nb_m = m > 0 ? (int)((m + kReduceRows - 1) / kReduceRows < kReduceBlocks ? (m + kReduceRows - 1) / kReduceRows : kReduceBlocks) : 0;
    const int nb_n = (int)((n + kReduceRows - 1) / kReduceRows < kReduceBlocks ? (n + kReduceRows - 1) / kReduceRows : kReduceBlocks);
    ReduceArgs<T> ra{};
    ra.m = m;
    ra.n = n;
    ra.ld = ld;
    ra.ncol = ncol;
    ra.nb_m = kReduceBlocks;  // partial layout stride: statistic s starts at s * kReduceBlocks * ld
    ra.nb_n = kReduceBlocks;
    ra.d_r = d.d_r;
    ra.d_c = d.d_c;
    ra.c = d.c;
    ra.xl = d.xl;
    ra.xu = d.xu;
    ra.l = d.l;
    ra.u = d.u;
    ra.col = d.col;
    ra.Xh = b.Xh;
    ra.DX = b.DX;
    ra.G = b.G;
    ra.X0 = b.X0;
    ra.X = b.X;
    ra.Yh = b.Yh;
    ra.DY = b.DY;
    ra.DYp = b.DYp;
    ra.Y0 = b.Y0;
    ra.Y = b.Y;
    ra.P0 = P0;
    ra.P1 = P1;
    ra.Q0 = Q0;
    ra.Q1 = Q1;
    ra.Q2 = Q2;
    ra.part = partials;
    ra.restart_to_output = d.restart_to_output;
    ra.robust_rc = d.robust_rc;
    const dim3 rblock(32, kReduceRows);
    if constexpr (kDf) {
        ReduceDfArgs<T> rd{};
        rd.m = m;
        rd.n = n;
        rd.ld = ld;
        rd.ncol = ncol;
        rd.dr = d.f_dr;
        rd.dc = d.f_dc;
        rd.idr = d.f_idr;
        rd.idc = d.f_idc;
        rd.c = d.f_c;
        rd.xl = d.f_xl;
        rd.xu = d.f_xu;
        rd.l = d.f_l;
        rd.u = d.f_u;
        rd.col = d.col;
        rd.Xh = b.Xh;
        rd.DX = b.DX;
        rd.X0 = b.X0;
        rd.X = b.X;
        rd.Yh = b.Yh;
        rd.DY = b.DY;
        rd.DYp = b.DYp;
        rd.Y0 = b.Y0;
        rd.Y = b.Y;
        rd.P0 = (const df*)P0;
        rd.P1 = (const df*)P1;
        rd.Q0 = (const df*)Q0;
        rd.Q1 = (const df*)Q1;
        rd.Q2 = (const df*)Q2;
        rd.part = partials;
        rd.restart_to_output = d.restart_to_output;
        rd.robust_rc = d.robust_rc;
        if (nb_m > 0) {
            k_reduce_m_df<T><<<dim3(nb_m, tiles), rblock, 0, s>>>(rd);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (d.At.n_long > 0)
            k_reduce_n_df<T><<<dim3(nb_n, tiles), rblock, 0, s>>>(rd);
        else
            k_check_n_df<T><<<dim3(nb_n, tiles), rblock, 0, s>>>(rd, d.At.rp, d.At.ci, d.At.v32, d.At.v32lo);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    } else {
        if (nb_m > 0) {
            k_reduce_rows_m<T><<<dim3(nb_m, tiles), rblock, 0, s>>>(ra);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        k_reduce_rows_n<T><<<dim3(nb_n, tiles), rblock, 0, s>>>(ra);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_colsum<<<dim3(tiles, kNumStats), dim3(32, 32), 0, s>>>(partials, nb_m, nb_n, ld, ncol, colsum);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    DecideArgs<T> da{};
    da.colsum = colsum;
    da.ld = ld;
    da.ncol = ncol;
    da.col = d.col;
    da.colp = colp;
    da.eta = d.eta;
    da.mnorm_sign = d.mnorm_sign;
    da.beta_s = d.beta_s;
    da.beta_n = d.beta_n;
    da.beta_a = d.beta_a;
    da.theta = d.theta;
    da.detect_inf = d.detect_inf;
    da.stall_checks = d.stall_checks;
    da.interval_len = interval_len;
    da.check_every = d.check_every;
    da.rec = rec;
    da.ctl = d.ctl;
    da.gcap = d.gcap;
    da.hal64 = d.hal64;
    da.hal32 = d.hal32;
    da.haldf = d.haldf;
    da.rscr = d.rscr;
    da.rtag = d.rtag;
    da.flags = d.flags;
    k_decide<T><<<1, kDecideThreads, 0, s>>>(da);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_restart_copy<T><<<blocks_for((size_t)n * ld, 256), 256, 0, s>>>(b.X, b.Xbar, b.X0, b.Xh, n, ld, ncol,
                                                                      d.restart_to_output, d.col.grp, d.ctl, d.flags);
    if (m > 0)
        k_restart_copy<T><<<blocks_for((size_t)m * ld, 256), 256, 0, s>>>(b.Y, nullptr, b.Y0, b.Yh, m, ld, ncol,
                                                                          d.restart_to_output, d.col.grp, d.ctl,
                                                                          d.flags);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], s)) != cudaSuccess) return e;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_admit(const CheckData& d, const IterData<T>& it, const IterBufs<T>& b, int ld, int c0, int count,
                         int group, int slot0, const lpb_lp_spec* specs_dev, const double* warm_x,
                         const double* warm_y, int64_t wsx, int64_t wsy, double c_norm_base, double b_norm,
                         double tol, double eps_inf, double tol_dual, int64_t max_iter, ColRecord* rec,
                         cudaStream_t s) {
    InitArgs<T> a{};
    a.m = d.m;
    a.n = d.n;
    a.ld = ld;
    a.c0 = c0;
    a.count = count;
    a.group = group;
    a.slot0 = slot0;
    a.specs = specs_dev;
    a.d_r = d.d_r;
    a.d_c = d.d_c;
    a.xl = d.xl;
    a.xu = d.xu;
    a.xls = it.xl;
    a.xus = it.xu;
    a.eta = d.eta;
    a.c_norm_base = c_norm_base;
    a.b_norm = b_norm;
    a.colp = it.col;
    a.colc = d.col;
    a.rec = rec;
    a.ctl = d.ctl;
    k_admit_group<<<1, 256, 0, s>>>(d.ctl, group, slot0, count, tol, eps_inf, tol_dual, (long long)max_iter,
                                    d.hal64, d.hal32, d.haldf, d.check_every);
    if (count <= 0) return cudaGetLastError();
    k_init_columns<T><<<(count + 255) / 256, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_init_iterates<T><<<blocks_for((size_t)(d.n + d.m) * count, 256), 256, 0, s>>>(a, b.Xbar, b.X0, b.Y, b.Y0, warm_x,
                                                                                    warm_y, wsx, wsy);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extract(const CheckData& d, const IterBufs<T>& b, int ld, const int* cols_dev,
                           double* const* outp_dev, int count, const double* xl_base, const double* xu_base,
                           cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int rows = d.n > d.m ? d.n : d.m;
    dim3 grid(blocks_for(rows, 256, 1024), count);
    k_extract<T><<<grid, 256, 0, s>>>(d.n, d.m, ld, cols_dev, outp_dev, count, d.d_r, d.d_c, xl_base, xu_base, d.col,
                                      b.Xh, b.Yh);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_compact(const IterBufs<T>& b, int n, int m, int ld, const int* src_dev, const int* dst_dev,
                           int count, ColParams<T> colp, ColCheck colc, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    k_compact_rows<T><<<blocks_for((size_t)(n + m) * count, 256), 256, 0, s>>>(b.Xbar, b.X0, b.Y, b.Y0, n, m, ld,
                                                                                src_dev, dst_dev, count);
    k_compact_cols<T><<<(count + 255) / 256, 256, 0, s>>>(colp, colc, src_dev, dst_dev, count);
    return cudaGetLastError();
}

namespace {

// state of column sc of the FP32 lane (the reflected point Xbar, the anchors,
// the dual iterate) -> column dc of the polish lane
template <typename TD>
__global__ void k_migrate_rows(const float* __restrict__ X, const float* __restrict__ X0,
                               const float* __restrict__ Y, const float* __restrict__ Y0, TD* __restrict__ DXs,
                               TD* __restrict__ DX0, TD* __restrict__ DY, TD* __restrict__ DY0, int n, int m,
                               int lds, int ldd, const int* __restrict__ sc, const int* __restrict__ dc, int count) {
    const size_t total = (size_t)(n + m) * count;
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int mv = (int)(p % count);
        const int row = (int)(p / count);
        if (row < n) {
            const size_t a = (size_t)row * lds + sc[mv], b = (size_t)row * ldd + dc[mv];
            DXs[b] = TD(X[a]);
            DX0[b] = TD(X0[a]);
        } else {
            const size_t a = (size_t)(row - n) * lds + sc[mv], b = (size_t)(row - n) * ldd + dc[mv];
            DY[b] = TD(Y[a]);
            DY0[b] = TD(Y0[a]);
        }
    }
}

// per-column data of the moved columns; the polish-precision parameters
// from the FP64 originals with the same formulas as k_init_columns and the
// column's current primal weight
template <typename TD>
__global__ void k_migrate_cols(ColCheck src, ColCheck dst, ColParams<TD> cp, const int* __restrict__ sc,
                               const int* __restrict__ dc, int count, int group, int slot_shift,
                               const double* __restrict__ d_c, double eta) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= count) return;
    const int s = sc[p], j = dc[p];
    const int kind = src.kind[s], var = src.var[s];
    const double w = src.w[s];
    dst.kind[j] = kind;
    dst.var[j] = var;
    dst.grp[j] = group;
    dst.lo[j] = src.lo[s];
    dst.hi[j] = src.hi[s];
    dst.c[j] = src.c[s];
    dst.w[j] = w;
    dst.slot[j] = src.slot[s] + slot_shift;
    dst.best[j] = src.best[s];
    dst.stall[j] = 0;
    double lo = 0.0, hi = 0.0, c = 0.0;
    if (kind == 1) {
        lo = src.lo[s] / d_c[var];
        hi = src.hi[s] / d_c[var];
    } else if (kind == 2) {
        c = d_c[var] * src.c[s];
    }
    cp.lo[j] = TD(lo);
    cp.hi[j] = TD(hi);
    cp.c[j] = TD(c);
    cp.tau[j] = TD(eta / w);
    cp.sigma[j] = TD(eta * w);
}

}  // namespace

template <typename TD>
cudaError_t launch_migrate(const CheckData& src, const IterBufs<float>& sb, int lds, const CheckData& dst,
                           const IterBufs<TD>& db, int ldd, ColParams<TD> dcolp, const int* sc_dev, const int* dc_dev,
                           int count, int group_dst, int slot_shift, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int n = src.n, m = src.m;
    k_migrate_rows<TD><<<blocks_for((size_t)(n + m) * count, 256), 256, 0, s>>>(
        sb.Xbar, sb.X0, sb.Y, sb.Y0, db.Xbar, db.X0, db.Y, db.Y0, n, m, lds, ldd, sc_dev, dc_dev, count);
    k_migrate_cols<TD><<<(count + 255) / 256, 256, 0, s>>>(src.col, dst.col, dcolp, sc_dev, dc_dev, count, group_dst,
                                                           slot_shift, src.d_c, src.eta);
    return cudaGetLastError();
}
template cudaError_t launch_migrate<double>(const CheckData&, const IterBufs<float>&, int, const CheckData&,
                                            const IterBufs<double>&, int, ColParams<double>, const int*, const int*,
                                            int, int, int, cudaStream_t);
template cudaError_t launch_migrate<dfloat>(const CheckData&, const IterBufs<float>&, int, const CheckData&,
                                            const IterBufs<dfloat>&, int, ColParams<dfloat>, const int*, const int*,
                                            int, int, int, cudaStream_t);

cudaError_t launch_group_moved(const CheckData& dst, int group, int slot0, cudaStream_t s) {
    k_group_moved<<<1, 256, 0, s>>>(dst.ctl, group, slot0, dst.hal64, dst.hal32, dst.haldf, dst.check_every);
    return cudaGetLastError();
}

#define LPB_INSTANTIATE(T)                                                                                        \
    template cudaError_t launch_check<T>(const CheckData&, const IterBufs<T>&, int, int, int, double*, double*,       \
                                         double*, double*, ColRecord*, ColParams<T>, cudaStream_t, cudaEvent_t*);     \
    template cudaError_t launch_admit<T>(const CheckData&, const IterData<T>&, const IterBufs<T>&, int, int, int,     \
                                         int, int, const lpb_lp_spec*, const double*, const double*, int64_t,         \
                                         int64_t, double, double, double, double, double, int64_t, ColRecord*,        \
                                         cudaStream_t);                                                               \
    template cudaError_t launch_extract<T>(const CheckData&, const IterBufs<T>&, int, const int*, double* const*,     \
                                           int, const double*, const double*, cudaStream_t);                          \
    template cudaError_t launch_compact<T>(const IterBufs<T>&, int, int, int, const int*, const int*, int,            \
                                           ColParams<T>, ColCheck, cudaStream_t);
LPB_INSTANTIATE(float)
LPB_INSTANTIATE(double)
LPB_INSTANTIATE(dfloat)

}  // namespace lpb
