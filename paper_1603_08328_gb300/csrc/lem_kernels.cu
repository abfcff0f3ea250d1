// CUDA kernels of local-expansion-move stereo (arXiv 1603.08328) for sm_103a.
//
// Layout in device memory (one pair; a batch concatenates its pairs):
//   L, R  : per pixel (R, G, B, x-gradient of gray), 0..255 scale, as float4
//           or as four FP16 / BF16 values
//   gst   : 3 float4 per pixel, guide mean mu_k and (Sigma_k + eU)^-1 (sym.)
//   wfw   : float4 per pixel, lambda * max(w_pq, eps), forward neighbours
//   lab   : float4 per pixel (a, b, c, phi_p(f_p)): label and cost cache
//   phiA  : float per pixel, phi_p(alpha) of the candidate being evaluated
//           (expansion regions of one group are disjoint, so one plane serves)
//   phiB  : float per pixel, the second candidate's phi in a two-CTA visit
//
// Regions of up to 5625 nodes (k_expand_group): one CTA evaluates, cuts and
// commits one expansion region; where a visit is two propagation candidates,
// a cluster of two CTAs computes the second data term alongside the first
// move.  The guided-filter data term is computed through the filtering
// region M as a strip pipeline in shared memory (raw cost rows -> vertical
// window sums -> horizontal window sums -> guided-filter coefficients -> their
// window means); the LE-BF data term sums bilateral weights times raw costs
// over each pixel's window.  The move graph is built in shared memory and cut
// by push-relabel with global relabelling.  Larger regions (k_expand_grid)
// run on several co-resident CTAs of a cooperative launch, with the graph in
// global memory and region barriers between rounds.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "lem_internal.h"

namespace lem {
namespace {

constexpr uint16_t kInf = 0xFFFF;
constexpr int kMaxVisit = 8;  // candidates per region visit held in shared memory

// 8-neighbourhood: k < 4 are the forward neighbours (1,0), (-1,1), (0,1), (1,1)
// (each unordered pair once); k >= 4 the opposite offsets.  Reverse of k is k^4.
__device__ __forceinline__ int dir_dx(int k) {
    const int d = k & 3;
    const int dx = (d == 0 || d == 3) ? 1 : (d == 1 ? -1 : 0);
    return k < 4 ? dx : -dx;
}
__device__ __forceinline__ int dir_dy(int k) {
    const int d = k & 3;
    const int dy = d == 0 ? 0 : 1;
    return k < 4 ? dy : -dy;
}
__device__ __forceinline__ float comp(const float4 &v, int d) {
    return d == 0 ? v.x : (d == 1 ? v.y : (d == 2 ? v.z : v.w));
}

// ---------------------------------------------------------------------------
// packed image pixels: float4, or four 16-bit floats (FP16 / BF16) converted
// to FP32 on load; all arithmetic is FP32
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 load_px(const void *base, size_t i, int fmt) {
    if (fmt == LEM_STORE_F32) return static_cast<const float4 *>(base)[i];
    const uint2 u = static_cast<const uint2 *>(base)[i];
    float2 a, b;
    if (fmt == LEM_STORE_F16) {
        a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    } else {
        a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
        b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    }
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store_px(void *base, size_t i, int fmt, float4 v) {
    if (fmt == LEM_STORE_F32) {
        static_cast<float4 *>(base)[i] = v;
        return;
    }
    uint2 u;
    if (fmt == LEM_STORE_F16) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        u.x = *reinterpret_cast<unsigned *>(&a);
        u.y = *reinterpret_cast<unsigned *>(&b);
    } else {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        u.x = *reinterpret_cast<unsigned *>(&a);
        u.y = *reinterpret_cast<unsigned *>(&b);
    }
    static_cast<uint2 *>(base)[i] = u;
}
__device__ __forceinline__ const void *px_offset(const void *base, long long off, int fmt) {
    return static_cast<const char *>(base) + off * (fmt == LEM_STORE_F32 ? 16 : 8);
}

// ---------------------------------------------------------------------------
// error-free transformations (never contracted into FMA: explicit _rn ops)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
__device__ __forceinline__ float two_prod(float a, float b, float &err) {
    const float p = __fmul_rn(a, b);
    err = __fmaf_rn(a, b, -p);
    return p;
}

// d_(u,v)(f1) - d_(u,v)(f2) with d_p(f) = a u + b v + c, in float-float so the
// result is accurate even for steep planes with large |c|.  The coefficient
// differences (dd_coef) are taken once per label pair and evaluated at any
// position (dd_eval).  Antisymmetric bit for bit: swapping f1 and f2 negates
// every intermediate exactly, so dd(f2, f1) == -dd(f1, f2).
struct DDCoef {
    float ah, al, bh, bl, ch, cl;
};
__device__ __forceinline__ DDCoef dd_coef(const float4 &f1, const float4 &f2) {
    DDCoef d;
    d.ah = two_sum(f1.x, -f2.x, d.al);
    d.bh = two_sum(f1.y, -f2.y, d.bl);
    d.ch = two_sum(f1.z, -f2.z, d.cl);
    return d;
}
__device__ __forceinline__ float dd_eval(const DDCoef &d, float u, float v) {
    float e1, e2, e3, e4;
    const float x1 = two_prod(d.ah, u, e1);
    const float x2 = two_prod(d.bh, v, e2);
    const float s1 = two_sum(x1, x2, e3);
    const float s2 = two_sum(s1, d.ch, e4);
    float lo = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, e4));
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fmul_rn(d.al, u), __fmul_rn(d.bl, v)), d.cl));
    return __fadd_rn(s2, lo);
}

// Q(wl min(pb, tau)) for psi-bar pb = |D1| + |D2| (Eq. smooth, Eq. smooth_phi),
// Q(x) = rne(S x)
__device__ __forceinline__ int q_of(float wl, float tau, float S, float D1, float D2) {
    const float pb = __fadd_rn(fabsf(D1), fabsf(D2));
    return __float2int_rn(__fmul_rn(__fmul_rn(wl, fminf(pb, tau)), S));
}

// Q(lambda psi_pq(f1, f2)) for the pair (p = (u1,v1), q = (u2,v2)) with weight
// wl = lambda max(w_pq, eps): psi-bar = |d_p(f1) - d_p(f2)| + |d_q(f2) - d_q(f1)|
// (Eq. smooth), truncated at tau_dis (Eq. smooth_phi); Q(x) = rne(S x).
// Symmetric bit for bit under swapping (f1 at p) <-> (f2 at q).
__device__ __forceinline__ int q_psi(float wl, float tau, float S, const float4 &f1, const float4 &f2, int u1,
                                     int v1, int u2, int v2) {
    const DDCoef d = dd_coef(f1, f2);
    return q_of(wl, tau, S, dd_eval(d, (float)u1, (float)v1), dd_eval(d, (float)u2, (float)v2));
}

__device__ __forceinline__ int q_cost(float phi, float S) { return __float2int_rn(__fmul_rn(phi, S)); }

// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014) and the random label arithmetic of the
// proposals, in FP64 with explicitly rounded operations so the candidate
// labels are bit-identical to a CPU evaluation of the same steps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long sm_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
struct Rng {
    unsigned long long s;
    __device__ double u01() {
        s += 0x9E3779B97F4A7C15ull;
        return __dmul_rn(__ull2double_rn(sm_mix(s) >> 11), 0x1.0p-53);
    }
};
__device__ __forceinline__ unsigned long long proposal_stream(unsigned long long seed, int iter, int level, int ci,
                                                              int cj, int prop) {
    unsigned long long s = sm_mix(seed);
    s = sm_mix(s ^ (unsigned long long)iter);
    s = sm_mix(s ^ (unsigned long long)level);
    s = sm_mix(s ^ (((unsigned long long)(unsigned)cj << 32) | (unsigned long long)(unsigned)ci));
    s = sm_mix(s ^ (unsigned long long)prop);
    return s;
}
__device__ __forceinline__ double dsq3(double x, double y, double z) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}
// uniform unit vector by rejection from the cube; (0,0,1) after 1000 misses
__device__ void unit_vec(Rng &g, double &x, double &y, double &z) {
    for (int t = 0; t < 1000; ++t) {
        const double a = __dsub_rn(__dmul_rn(2.0, g.u01()), 1.0);
        const double b = __dsub_rn(__dmul_rn(2.0, g.u01()), 1.0);
        const double c = __dsub_rn(__dmul_rn(2.0, g.u01()), 1.0);
        const double s = dsq3(a, b, c);
        if (s > 1.0 || s == 0.0) continue;
        const double l = __dsqrt_rn(s);
        x = __ddiv_rn(a, l);
        y = __ddiv_rn(b, l);
        z = __ddiv_rn(c, l);
        return;
    }
    x = 0.0;
    y = 0.0;
    z = 1.0;
}
// plane through (u, v, z0) with unit normal n: a = -nx/nz, b = -ny/nz,
// c = (nx u + ny v + nz z0)/nz
__device__ __forceinline__ float4 plane_from(double nx, double ny, double nz, int u, int v, double z0) {
    const double c = __ddiv_rn(__dadd_rn(__dadd_rn(__dmul_rn(nx, (double)u), __dmul_rn(ny, (double)v)),
                                         __dmul_rn(nz, z0)),
                               nz);
    return make_float4(__double2float_rn(__ddiv_rn(-nx, nz)), __double2float_rn(__ddiv_rn(-ny, nz)),
                       __double2float_rn(c), 0.f);
}

// Candidate of one proposal of Algorithm 2 from the current label map.
__device__ float4 propose(const float4 *lab, int W, unsigned long long stream, int cx0, int cy0, int cw, int chh,
                          bool perturb, double rd, double rn, double dmin, double dmax) {
    Rng g{stream};
    const int n = cw * chh;
    int k = (int)__dmul_rn(g.u01(), (double)n);
    if (k >= n) k = n - 1;
    const int ru = cx0 + k % cw, rv = cy0 + k / cw;
    const float4 f = lab[(size_t)rv * W + ru];
    if (!perturb) return make_float4(f.x, f.y, f.z, 0.f);
    const double a = f.x, b = f.y, c = f.z;
    const double d = __dadd_rn(__dadd_rn(__dmul_rn(a, (double)ru), __dmul_rn(b, (double)rv)), c);
    const double len = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), 1.0));
    const double n0 = __ddiv_rn(-a, len), n1 = __ddiv_rn(-b, len), n2 = __ddiv_rn(1.0, len);
    double dp = __dadd_rn(d, __dmul_rn(rd, __dsub_rn(__dmul_rn(2.0, g.u01()), 1.0)));
    if (dp < dmin) dp = dmin;
    if (dp > dmax) dp = dmax;
    double m0 = n0, m1 = n1, m2 = n2;
    for (int t = 0; t < 64; ++t) {
        double vx, vy, vz;
        unit_vec(g, vx, vy, vz);
        double q0 = __dadd_rn(n0, __dmul_rn(rn, vx));
        double q1 = __dadd_rn(n1, __dmul_rn(rn, vy));
        double q2 = __dadd_rn(n2, __dmul_rn(rn, vz));
        const double ql = __dsqrt_rn(dsq3(q0, q1, q2));
        if (ql == 0.0) continue;
        q0 = __ddiv_rn(q0, ql);
        q1 = __ddiv_rn(q1, ql);
        q2 = __ddiv_rn(q2, ql);
        if (fabs(q2) < 1e-3) continue;
        m0 = q0;
        m1 = q1;
        m2 = q2;
        break;
    }
    return plane_from(m0, m1, m2, ru, rv, dp);
}


// ---------------------------------------------------------------------------
// RANSAC proposer (Algorithm 2, RANSAC proposal): LO-RANSAC plane fit to the current
// disparities of the centre cell, computed by the whole CTA.  The steps and their
// rounding are the oracle's: disparities on the 2^-20 grid, 32 hypotheses through
// three pixels drawn from the proposal's stream, 1 px inliers, the best (first on
// ties) refined twice by least squares with exact integer sums and Cramer's rule
// in FP64 with one rounding per operation, cell-relative coordinates.
// ---------------------------------------------------------------------------
constexpr int kRansacHyp = 32;
constexpr int kRansacLo = 2;
constexpr int kRansacMaxCell = kRansacSmemCell;
constexpr double kRansacQ = 1048576.0;

struct RansacSmem {
    long long dq[kRansacMaxCell];
    int id[kRansacHyp * 3];
    double pl[kRansacHyp * 3];
    int cnt[kRansacHyp];
    int ok[kRansacHyp];
    unsigned long long sums[10];
    double best[3];
    int state;  // 0: no valid hypothesis, 1: plane in best
};

__device__ __forceinline__ bool ransac_inlier(long long dq, int x, int y, double a, double b, double c) {
    const double r = __dsub_rn(__ddiv_rn(__ll2double_rn(dq), kRansacQ),
                               __dadd_rn(__dadd_rn(__dmul_rn(a, (double)x), __dmul_rn(b, (double)y)), c));
    return fabs(r) <= 1.0;
}

// all threads of the CTA; *out written by thread 0; ends with a barrier.
//   dq: cw * chh quantised disparities of the cell (R->dq for cells of at most
//       kRansacMaxCell pixels, else a global scratch of the CTA)
__device__ void ransac_cta(const float4 *lab, int W, unsigned long long stream, int cx0, int cy0, int cw, int chh,
                           RansacSmem *R, long long *dq, float4 *out) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    const int n = cw * chh;
    for (int k = tid; k < n; k += nt) {
        const int x = k % cw, y = k / cw, u = cx0 + x, v = cy0 + y;
        const float4 f = lab[(size_t)v * W + u];
        const double d = __dadd_rn(__dadd_rn(__dmul_rn((double)f.x, (double)u), __dmul_rn((double)f.y, (double)v)),
                                   (double)f.z);
        dq[k] = __double2ll_rn(__dmul_rn(d, kRansacQ));
    }
    if (tid == 0) {
        Rng g{stream};
        for (int j = 0; j < 3 * kRansacHyp; ++j) {
            int k = (int)__dmul_rn(g.u01(), (double)n);
            if (k >= n) k = n - 1;
            R->id[j] = k;
        }
    }
    __syncthreads();
    if (tid < kRansacHyp) {
        const int i0 = R->id[3 * tid], i1 = R->id[3 * tid + 1], i2 = R->id[3 * tid + 2];
        int ok = 0;
        if (i0 != i1 && i0 != i2 && i1 != i2) {
            const long long x0 = i0 % cw, y0 = i0 / cw, x1 = i1 % cw, y1 = i1 / cw, x2 = i2 % cw, y2 = i2 / cw;
            const long long du1 = x1 - x0, dv1 = y1 - y0, du2 = x2 - x0, dv2 = y2 - y0;
            const long long det = du1 * dv2 - du2 * dv1;
            if (det != 0) {
                const long long dd1 = dq[i1] - dq[i0], dd2 = dq[i2] - dq[i0];
                const long long na = dd1 * dv2 - dd2 * dv1, nb = du1 * dd2 - du2 * dd1;
                const double den = __dmul_rn(__ll2double_rn(det), kRansacQ);
                const double a = __ddiv_rn(__ll2double_rn(na), den), b = __ddiv_rn(__ll2double_rn(nb), den);
                const double c = __dsub_rn(__dsub_rn(__ddiv_rn(__ll2double_rn(dq[i0]), kRansacQ),
                                                     __dmul_rn(a, (double)x0)),
                                           __dmul_rn(b, (double)y0));
                R->pl[3 * tid] = a;
                R->pl[3 * tid + 1] = b;
                R->pl[3 * tid + 2] = c;
                ok = 1;
            }
        }
        R->ok[tid] = ok;
    }
    __syncthreads();
    for (int hy = warp; hy < kRansacHyp; hy += nwarp) {
        int c = 0;
        if (R->ok[hy]) {
            const double a = R->pl[3 * hy], b = R->pl[3 * hy + 1], cc = R->pl[3 * hy + 2];
            for (int k = lane; k < n; k += 32) c += ransac_inlier(dq[k], k % cw, k / cw, a, b, cc) ? 1 : 0;
        }
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) R->cnt[hy] = R->ok[hy] ? c : -1;
    }
    __syncthreads();
    if (tid == 0) {
        int best = -1, bc = -1;
        for (int hy = 0; hy < kRansacHyp; ++hy)
            if (R->cnt[hy] > bc) {
                bc = R->cnt[hy];
                best = hy;
            }
        if (bc < 0) {
            R->state = 0;
            const int k = R->id[0];
            const float4 f = lab[(size_t)(cy0 + k / cw) * W + cx0 + k % cw];
            *out = make_float4(f.x, f.y, f.z, 0.f);
        } else {
            R->state = 1;
            R->best[0] = R->pl[3 * best];
            R->best[1] = R->pl[3 * best + 1];
            R->best[2] = R->pl[3 * best + 2];
        }
    }
    __syncthreads();
    if (R->state == 0) return;  // (uniform) the barrier above published *out
    for (int it = 0; it < kRansacLo; ++it) {
        if (tid < 10) R->sums[tid] = 0ull;
        __syncthreads();
        const double a = R->best[0], b = R->best[1], c = R->best[2];
        long long s[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int k = tid; k < n; k += nt) {
            const long long x = k % cw, y = k / cw, dqk = dq[k];
            if (!ransac_inlier(dqk, (int)x, (int)y, a, b, c)) continue;
            s[0] += x * x;
            s[1] += x * y;
            s[2] += x;
            s[3] += y * y;
            s[4] += y;
            s[5] += 1;
            s[6] += x * dqk;
            s[7] += y * dqk;
            s[8] += dqk;
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            long long vq = s[q];
            for (int o = 16; o > 0; o >>= 1) vq += __shfl_xor_sync(0xffffffffu, vq, o);
            if (lane == 0 && vq != 0) atomicAdd(&R->sums[q], (unsigned long long)vq);
        }
        __syncthreads();
        if (tid == 0) {
            R->sums[9] = 0ull;  // 1: stop refining
            if ((long long)R->sums[5] < 3) {
                R->sums[9] = 1ull;
            } else {
                const double m00 = __ll2double_rn((long long)R->sums[0]), m01 = __ll2double_rn((long long)R->sums[1]);
                const double m02 = __ll2double_rn((long long)R->sums[2]), m11 = __ll2double_rn((long long)R->sums[3]);
                const double m12 = __ll2double_rn((long long)R->sums[4]), m22 = __ll2double_rn((long long)R->sums[5]);
                const double r0 = __ll2double_rn((long long)R->sums[6]), r1 = __ll2double_rn((long long)R->sums[7]);
                const double r2 = __ll2double_rn((long long)R->sums[8]);
                const double c00 = __dsub_rn(__dmul_rn(m11, m22), __dmul_rn(m12, m12));
                const double c01 = __dsub_rn(__dmul_rn(m01, m22), __dmul_rn(m12, m02));
                const double c02 = __dsub_rn(__dmul_rn(m01, m12), __dmul_rn(m11, m02));
                const double det = __dadd_rn(__dsub_rn(__dmul_rn(m00, c00), __dmul_rn(m01, c01)), __dmul_rn(m02, c02));
                if (det == 0.0) {
                    R->sums[9] = 1ull;
                } else {
                    const double t1 = __dsub_rn(__dmul_rn(r1, m22), __dmul_rn(m12, r2));
                    const double t2 = __dsub_rn(__dmul_rn(r1, m12), __dmul_rn(m11, r2));
                    const double t3 = __dsub_rn(__dmul_rn(m01, r2), __dmul_rn(r1, m02));
                    const double t4 = __dsub_rn(__dmul_rn(m11, r2), __dmul_rn(r1, m12));
                    const double da = __dadd_rn(__dsub_rn(__dmul_rn(r0, c00), __dmul_rn(m01, t1)), __dmul_rn(m02, t2));
                    const double db = __dadd_rn(__dsub_rn(__dmul_rn(m00, t1), __dmul_rn(r0, c01)), __dmul_rn(m02, t3));
                    const double dc = __dadd_rn(__dsub_rn(__dmul_rn(m00, t4), __dmul_rn(m01, t3)), __dmul_rn(r0, c02));
                    const double den = __dmul_rn(det, kRansacQ);
                    R->best[0] = __ddiv_rn(da, den);
                    R->best[1] = __ddiv_rn(db, den);
                    R->best[2] = __ddiv_rn(dc, den);
                }
            }
        }
        __syncthreads();
        if (R->sums[9]) break;  // (uniform)
    }
    if (tid == 0) {
        const double a = R->best[0], b = R->best[1];
        const double c = __dsub_rn(__dsub_rn(R->best[2], __dmul_rn(a, (double)cx0)), __dmul_rn(b, (double)cy0));
        *out = make_float4(__double2float_rn(a), __double2float_rn(b), __double2float_rn(c), 0.f);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// K0: packing, contrast weights, guide statistics, random init
// ---------------------------------------------------------------------------
__device__ __forceinline__ int gray1000(const uint8_t *c) { return 299 * c[0] + 587 * c[1] + 114 * c[2]; }

__global__ void k_preprocess(const uint8_t *left, int64_t ls, const uint8_t *right, int64_t rs, int H, int W,
                             float lambda, float eps_w, float gamma, void *Lp, void *Rp, int fmt, float4 *wfw) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const uint8_t *lr = left + (size_t)y * ls, *rr = right + (size_t)y * rs;
    const int xm = max(x - 1, 0), xp = min(x + 1, W - 1);
    // BT.601 gray x 1000 is an exact integer; the [-0.5 0 0.5] gradient is
    // then one correctly rounded division
    const float gl = (float)(gray1000(lr + 3 * xp) - gray1000(lr + 3 * xm)) / 2000.0f;
    const float gr = (float)(gray1000(rr + 3 * xp) - gray1000(rr + 3 * xm)) / 2000.0f;
    const size_t p = (size_t)y * W + x;
    store_px(Lp, p, fmt, make_float4(lr[3 * x], lr[3 * x + 1], lr[3 * x + 2], gl));
    store_px(Rp, p, fmt, make_float4(rr[3 * x], rr[3 * x + 1], rr[3 * x + 2], gr));
    float w[4];
    for (int d = 0; d < 4; ++d) {
        const int qx = x + dir_dx(d), qy = y + dir_dy(d);
        w[d] = 0.f;
        if (qx < 0 || qx >= W || qy >= H) continue;
        const uint8_t *a = lr + 3 * x, *b = left + (size_t)qy * ls + 3 * qx;
        const int l1 = abs((int)a[0] - (int)b[0]) + abs((int)a[1] - (int)b[1]) + abs((int)a[2] - (int)b[2]);
        const float wv = expf(-(float)l1 / gamma);
        w[d] = lambda * fmaxf(wv, eps_w);
    }
    wfw[p] = make_float4(w[0], w[1], w[2], w[3]);
}

// Guide statistics over the clipped window W'_k: exact integer window sums of
// the 8-bit colours, so N^2 255^2 Sigma_k = N S2 - S1 S1^T is exact in int64.
// (Sigma_k + eU)^-1 by the adjugate in FP32; when the Frobenius condition
// estimate exceeds cond_fp64 the inverse is redone in FP64 from the exact sums.
__global__ void k_guide_stats(const uint8_t *left, int64_t ls, int H, int W, int r, double eps, double cond_fp64,
                              float4 *gst, int *n_fp64) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const int x0 = max(0, x - r), x1 = min(W - 1, x + r), y0 = max(0, y - r), y1 = min(H - 1, y + r);
    int s1[3] = {0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0};
    for (int yy = y0; yy <= y1; ++yy) {
        const uint8_t *row = left + (size_t)yy * ls;
        for (int xx = x0; xx <= x1; ++xx) {
            const int r0 = row[3 * xx], g0 = row[3 * xx + 1], b0 = row[3 * xx + 2];
            s1[0] += r0;
            s1[1] += g0;
            s1[2] += b0;
            s2[0] += r0 * r0;
            s2[1] += r0 * g0;
            s2[2] += r0 * b0;
            s2[3] += g0 * g0;
            s2[4] += g0 * b0;
            s2[5] += b0 * b0;
        }
    }
    const long long N = (long long)(x1 - x0 + 1) * (y1 - y0 + 1);
    const int ii[6] = {0, 0, 0, 1, 1, 2}, jj[6] = {0, 1, 2, 1, 2, 2};
    long long num[6];
    for (int k = 0; k < 6; ++k) num[k] = N * (long long)s2[k] - (long long)s1[ii[k]] * (long long)s1[jj[k]];
    const float den = (float)((double)N * (double)N * 65025.0);
    float m[6];
    for (int k = 0; k < 6; ++k) m[k] = (float)num[k] / den;
    m[0] += (float)eps;
    m[3] += (float)eps;
    m[5] += (float)eps;
    // adjugate of [[m0 m1 m2] [m1 m3 m4] [m2 m4 m5]]
    float c00 = m[3] * m[5] - m[4] * m[4], c01 = m[2] * m[4] - m[1] * m[5], c02 = m[1] * m[4] - m[2] * m[3];
    float c11 = m[0] * m[5] - m[2] * m[2], c12 = m[1] * m[2] - m[0] * m[4], c22 = m[0] * m[3] - m[1] * m[1];
    float det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    float inv[6] = {c00 / det, c01 / det, c02 / det, c11 / det, c12 / det, c22 / det};
    float nm = 0.f, ni = 0.f;
    for (int k = 0; k < 6; ++k) {
        const float wgt = (k == 0 || k == 3 || k == 5) ? 1.f : 2.f;
        nm += wgt * m[k] * m[k];
        ni += wgt * inv[k] * inv[k];
    }
    const float cond = sqrtf(nm) * sqrtf(ni);
    if (!(cond <= (float)cond_fp64)) {
        double d[6];
        const double dd = (double)N * (double)N * 65025.0;
        for (int k = 0; k < 6; ++k) d[k] = (double)num[k] / dd;
        d[0] += eps;
        d[3] += eps;
        d[5] += eps;
        const double e00 = d[3] * d[5] - d[4] * d[4], e01 = d[2] * d[4] - d[1] * d[5],
                     e02 = d[1] * d[4] - d[2] * d[3];
        const double e11 = d[0] * d[5] - d[2] * d[2], e12 = d[1] * d[2] - d[0] * d[4],
                     e22 = d[0] * d[3] - d[1] * d[1];
        const double dt = d[0] * e00 + d[1] * e01 + d[2] * e02;
        inv[0] = (float)(e00 / dt);
        inv[1] = (float)(e01 / dt);
        inv[2] = (float)(e02 / dt);
        inv[3] = (float)(e11 / dt);
        inv[4] = (float)(e12 / dt);
        inv[5] = (float)(e22 / dt);
        atomicAdd(n_fp64, 1);
    }
    const float n255 = 255.f * (float)N;
    const size_t p = (size_t)y * W + x;
    gst[3 * p + 0] = make_float4((float)s1[0] / n255, (float)s1[1] / n255, (float)s1[2] / n255, inv[0]);
    gst[3 * p + 1] = make_float4(inv[1], inv[2], inv[3], inv[4]);
    gst[3 * p + 2] = make_float4(inv[5], 0.f, 0.f, 0.f);
}

// Random initial labels (Sec. 3.4): z0 uniform in [dmin, dmax], unit normal by
// rejection (redrawn while |n_z| < 1e-3, at most 64 tries, else (0,0,1)).
__global__ void k_init_labels(int H, int W, unsigned long long seed, double dmin, double dmax, float4 *lab) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    Rng g{sm_mix(sm_mix(seed ^ 0x5851F42D4C957F2Dull) ^ (unsigned long long)((long long)y * W + x))};
    const double z0 = __dadd_rn(dmin, __dmul_rn(__dsub_rn(dmax, dmin), g.u01()));
    double nx = 0.0, ny = 0.0, nz = 1.0;
    for (int t = 0; t < 64; ++t) {
        double a, b, c;
        unit_vec(g, a, b, c);
        if (fabs(c) < 1e-3) continue;
        nx = a;
        ny = b;
        nz = c;
        break;
    }
    lab[(size_t)y * W + x] = plane_from(nx, ny, nz, x, y, z0);
}

// ---------------------------------------------------------------------------
// A3 + A4: data term of one label over one region, through M
// ---------------------------------------------------------------------------
// sum of count values base[0], base[stride], ... with four independent partial sums
// The window sums of the guided filter keep four channels of a pixel together
// (one float4 per pixel), so one 16-byte shared load feeds four sums; every
// channel is summed exactly as a scalar sum would be.
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ float4 sub4(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
// sum of `count` values at base, base + stride, ... in four interleaved partial
// sums, ((a0 + a1) + (a2 + a3)) per channel
__device__ __forceinline__ float4 strided_sum4(const float4 *base, int stride, int count) {
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int i = 0;
    for (; i + 4 <= count; i += 4) {
        a0 = add4(a0, base[i * stride]);
        a1 = add4(a1, base[(i + 1) * stride]);
        a2 = add4(a2, base[(i + 2) * stride]);
        a3 = add4(a3, base[(i + 3) * stride]);
    }
    for (; i < count; ++i) a0 = add4(a0, base[i * stride]);
    return add4(add4(a0, a1), add4(a2, a3));
}
__device__ __forceinline__ int ring_next(int s, int RS) { return s + 1 == RS ? 0 : s + 1; }
// the same over `count` consecutive rows of a ring of RS rows (row pitch rs) from
// slot s0, with the same association as strided_sum4 over those rows in order
// (wherever the ring wraps)
__device__ __forceinline__ float4 ring_sum4(const float4 *base, int rs, int RS, int s0, int count) {
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0, a2 = a0, a3 = a0;
    int i = 0, s = s0;
    for (; i + 4 <= count; i += 4) {
        a0 = add4(a0, base[s * rs]);
        s = ring_next(s, RS);
        a1 = add4(a1, base[s * rs]);
        s = ring_next(s, RS);
        a2 = add4(a2, base[s * rs]);
        s = ring_next(s, RS);
        a3 = add4(a3, base[s * rs]);
        s = ring_next(s, RS);
    }
    for (; i < count; ++i) {
        a0 = add4(a0, base[s * rs]);
        s = ring_next(s, RS);
    }
    return add4(add4(a0, a1), add4(a2, a3));
}

// Thread layout of one pipeline stage over an R x C item grid: threads form
// rows of min(C, nt) columns; the (single) division happens once per stage.
// raw cost (Eq. photofunc) from the colour and gradient differences, each
// operation rounded once in a fixed order, so every kernel that inlines it gets
// the same bits whatever the compiler fuses around it
__device__ __forceinline__ float rho_mix(float col, float gd, const KParams &kp, float oma) {
    return __fmaf_rn(oma, fminf(col, kp.tau_col), __fmul_rn(kp.alpha_grad, fminf(gd, kp.tau_grad)));
}

struct Grid2 {
    int tc, tr, cpr, rpp;
    __device__ Grid2(int C) {
        cpr = min(C, (int)blockDim.x);
        rpp = blockDim.x / cpr;
        tc = threadIdx.x % cpr;
        tr = threadIdx.x / cpr;
    }
};

// Warp offset of row y relative to column x0: Q(y) = (1 - a) x0 - b y - c, with
// 1 - a = sh + sl in float-float, kept as integer I + fraction F in [0, 1).
__device__ __forceinline__ void row_offset(float sh, float sl, float lb, float lc, int x0, int y, int &I, float &F) {
    float e1, e2, e3, e4;
    const float p = two_prod(sh, (float)x0, e1);
    const float q = two_prod(lb, (float)y, e2);
    const float t1 = two_sum(p, -q, e3);
    const float t2 = two_sum(t1, -lc, e4);
    const float lo = __fadd_rn(__fadd_rn(__fsub_rn(e1, e2), __fadd_rn(e3, e4)), __fmul_rn(sl, (float)x0));
    const float th = fminf(fmaxf(t2, -1.0e9f), 1.0e9f);
    const float fl = floorf(th);
    F = __fadd_rn(__fsub_rn(th, fl), lo);
    I = (int)fl;
    if (F < 0.f) {
        F += 1.f;
        I -= 1;
    } else if (F >= 1.f) {
        F -= 1.f;
        I += 1;
    }
}

// phi_p(f) for p in [Rx0, Rx0+Rw) x [Ry0, Ry0+Rh); out[(py-Ry0)*pitch + px-Rx0].
// Guided-filter aggregation (Eq. gf): mean over the windows W'_k containing p
// of a_k . I_p + b_k, a_k = (Sigma_k+eU)^-1 (mean(I rho) - mu_k mean(rho)),
// b_k = mean(rho) - a_k . mu_k, every window clipped to the image and
// normalised by its pixel count.  The guide is centred on the colour at the
// region centre (the filter is invariant to a constant shift of the guide),
// which keeps the covariance differences small in flat areas.
//
// Strip pipeline: M rows enter a ring of T + 2r' rows of the four channels
// (rho, (I - c) rho), kept together per pixel as one float4 so that a 16-byte
// shared load serves the four window sums; every T rows of K (R grown by r') get vertical then
// horizontal window sums and their a_k, b_k, which enter a second ring of
// T + 2r' + 4 rows; every T rows of R get the window means of a_k, b_k and phi.
// Every sliding window sum restarts at rows Ky0 + 4m, Ry0 + 4m and columns
// Kx0 + 8m, Rx0 + 4m (at most 27, or 35 for the 8-column runs, terms per sum)
// and is accumulated by one thread in a fixed order, so with T a multiple of 4
// the result does not depend on T or on the CTA size.
__device__ void region_unary_gf(const DevPlanes &P, const KParams &kp, int Rx0, int Ry0, int Rw, int Rh, float la,
                             float lb, float lc, float *sm, float *out, int pitch) {
    const int H = P.H, W = P.W, r = kp.r, T = kp.T;
    const int Mx0 = max(0, Rx0 - 2 * r), Mx1 = min(W, Rx0 + Rw + 2 * r);
    const int My0 = max(0, Ry0 - 2 * r), My1 = min(H, Ry0 + Rh + 2 * r);
    const int Kx0 = max(0, Rx0 - r), Kx1 = min(W, Rx0 + Rw + r);
    const int Ky0 = max(0, Ry0 - r), Ky1 = min(H, Ry0 + Rh + r);
    const int Mw = Mx1 - Mx0, Kw = Kx1 - Kx0;
    const int RS = T + 2 * r, RSA = RS + 4;
    // four channels per pixel in one float4 (16 bytes)
    float4 *Xr = reinterpret_cast<float4 *>(sm);  // [RS][Mw]  (rho, (I - c) rho) of M rows (ring)
    float4 *Vb = Xr + (size_t)RS * Mw;            // [T][Mw]   vertical sums (also [T][Kw])
    float4 *Bb = Vb + (size_t)T * Mw;             // [T][Kw]   box sums      (also [T][Rw])
    float4 *ABr = Bb + (size_t)T * Kw;            // [RSA][Kw] (a_k, b_k) of K rows (ring)

    const int fmt = P.fmt;
    const float4 cen4 = load_px(P.L, (size_t)(Ry0 + Rh / 2) * W + (Rx0 + Rw / 2), fmt);
    const float inv255 = 1.0f / 255.0f;
    const float cr = cen4.x * inv255, cg = cen4.y * inv255, cb = cen4.z * inv255;
    // warp s' = s - (a s_u + b s_v + c): u' = x - d = Q(y) + (1-a)(x - Rx0) with
    // Q(y) = (1-a) Rx0 - b y - c kept as integer + fraction in float-float
    float sl;
    const float sh = two_sum(1.0f, -la, sl);
    const float oma = 1.0f - kp.alpha_grad;

    // stage layouts (fixed for the call)
    const Grid2 gM(Mw), gK(Kw), gR(Rw), gV(Mw), gV2(Kw);
    const int nchK = (Kw + 7) >> 3, nchR = (Rw + 3) >> 2;
    const Grid2 gH(nchK), gH2(nchR);

    int mNext = My0, kNext = Ky0;
    int mSlot = 0;  // ring slot of row mNext in Xr
    int kSlot = 0;  // ring slot of row kNext in ABr
    for (int p0 = Ry0; p0 < Ry0 + Rh; p0 += T) {
        const int p1 = min(Ry0 + Rh, p0 + T);
        // K rows are computed in chunks that start at Ky0 + 4m: the rows needed
        // up to p1 + r, rounded up to that grid (at most 3 rows ahead)
        const int kNeed = min(Ky1, Ky0 + ((p1 + r - Ky0 + 3) & ~3));
        while (kNext < kNeed) {
            const int k0 = kNext, k1 = min(kNeed, k0 + T);
            const int mNeed = min(My1, k1 + r);
            if (mNext < mNeed) {
                const int nrow = mNeed - mNext;
                if (gM.tr < gM.rpp) {
                    for (int i = gM.tr; i < nrow; i += gM.rpp) {
                        const int y = mNext + i;
                        int slot = mSlot + i;
                        if (slot >= RS) slot -= RS;
                        // the row's warp offset, by every thread of the row (no barrier)
                        int Ib;
                        float Fb;
                        row_offset(sh, sl, lb, lc, Rx0, y, Ib, Fb);
                        const size_t rowb = (size_t)y * W;
                        float4 *o = Xr + (size_t)slot * Mw;
                        for (int xc = gM.tc; xc < Mw; xc += gM.cpr) {
                            const int x = Mx0 + xc;
                            const float4 l = load_px(P.L, rowb + x, fmt);
                            const float dx = (float)(x - Rx0);
                            const float g = __fmaf_rn(sh, dx, __fmaf_rn(sl, dx, Fb));
                            const float gf = floorf(g);
                            float t = g - gf;
                            int i0 = Ib + (int)gf;
                            if (i0 < 0) {
                                i0 = 0;
                                t = 0.f;
                            } else if (i0 >= W - 1) {
                                i0 = W - 1;
                                t = 0.f;
                            }
                            const int i1 = min(i0 + 1, W - 1);
                            const float4 r0 = load_px(P.R, rowb + i0, fmt), r1 = load_px(P.R, rowb + i1, fmt);
                            const float rr = fmaf(t, r1.x - r0.x, r0.x);
                            const float rg = fmaf(t, r1.y - r0.y, r0.y);
                            const float rb = fmaf(t, r1.z - r0.z, r0.z);
                            const float rd = fmaf(t, r1.w - r0.w, r0.w);
                            const float col = fabsf(l.x - rr) + fabsf(l.y - rg) + fabsf(l.z - rb);
                            const float gd = fabsf(l.w - rd);
                            const float rho = rho_mix(col, gd, kp, oma);
                            o[xc] = make_float4(rho, __fmul_rn(__fmaf_rn(l.x, inv255, -cr), rho),
                                                __fmul_rn(__fmaf_rn(l.y, inv255, -cg), rho),
                                                __fmul_rn(__fmaf_rn(l.z, inv255, -cb), rho));
                        }
                    }
                }
                mSlot += nrow;
                if (mSlot >= RS) mSlot -= RS;
                mNext = mNeed;
                __syncthreads();
            }
            // vertical window sums of the 4 channels for K rows [k0, k1): item =
            // M column by group of 4 consecutive output rows
            {
                const int ng = (k1 - k0 + 3) >> 2;
                const int rs = Mw;
                if (gV.tr < gV.rpp) {
                    for (int cc = gV.tc; cc < Mw; cc += gV.cpr) {
                        const float4 *X = Xr + cc;
                        float4 *V = Vb + cc;
                        for (int grp = gV.tr; grp < ng; grp += gV.rpp) {
                            const int ky0 = k0 + 4 * grp, ky1 = min(k1, ky0 + 4);
                            const int ylo = max(0, ky0 - r), yhi = min(H - 1, ky0 + r);
                            // slot of row ylo: rows mNext - RS .. mNext - 1 are in the ring
                            int sIn = mSlot - (mNext - ylo);
                            if (sIn < 0) sIn += RS;
                            float4 sm = ring_sum4(X, rs, RS, sIn, yhi - ylo + 1);
                            V[(ky0 - k0) * rs] = sm;
                            int sA = sIn + (yhi - ylo + 1);  // slot of row yhi + 1
                            if (sA >= RS) sA -= RS;
                            int sO = sIn;                    // slot of row ylo
                            for (int ky = ky0 + 1; ky < ky1; ++ky) {
                                if (ky + r <= H - 1) {
                                    sm = add4(sm, X[sA * rs]);
                                    sA = ring_next(sA, RS);
                                }
                                if (ky - r - 1 >= 0) {
                                    sm = sub4(sm, X[sO * rs]);
                                    sO = ring_next(sO, RS);
                                }
                                V[(ky - k0) * rs] = sm;
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // horizontal window sums at K columns, 8 outputs (of 4 channels) per item
            if (gH.tr < gH.rpp) {
                for (int chunk = gH.tc; chunk < nchK; chunk += gH.cpr) {
                    const int kx0 = Kx0 + chunk * 8, kx1 = min(Kx1, kx0 + 8);
                    const int xlo = max(0, kx0 - r), xhi = min(W - 1, kx0 + r);
                    for (int row = gH.tr; row < k1 - k0; row += gH.rpp) {
                        const float4 *V = Vb + row * Mw - Mx0;
                        float4 *B = Bb + row * Kw - Kx0;
                        float4 sm = strided_sum4(V + xlo, 1, xhi - xlo + 1);
                        B[kx0] = sm;
                        for (int kx = kx0 + 1; kx < kx1; ++kx) {
                            if (kx + r <= W - 1) sm = add4(sm, V[kx + r]);
                            if (kx - r - 1 >= 0) sm = sub4(sm, V[kx - r - 1]);
                            B[kx] = sm;
                        }
                    }
                }
            }
            __syncthreads();
            // guided-filter coefficients a_k, b_k for K rows [k0, k1)
            if (gK.tr < gK.rpp) {
                for (int row = gK.tr; row < k1 - k0; row += gK.rpp) {
                    const int ky = k0 + row;
                    const int ny = min(H - 1, ky + r) - max(0, ky - r) + 1;
                    int slot = kSlot + row;
                    if (slot >= RSA) slot -= RSA;
                    float4 *A = ABr + slot * Kw;
                    const float4 *B = Bb + row * Kw;
                    const float4 *G = P.gst + 3 * ((size_t)ky * W + Kx0);
                    for (int col = gK.tc; col < Kw; col += gK.cpr) {
                        const int kx = Kx0 + col;
                        const float n = (float)((min(W - 1, kx + r) - max(0, kx - r) + 1) * ny);
                        const float inv = 1.0f / n;
                        const float4 bs = B[col];
                        const float mr = bs.x * inv;
                        const float4 g0 = G[3 * col], g1 = G[3 * col + 1], g2 = G[3 * col + 2];
                        const float u0 = g0.x - cr, u1 = g0.y - cg, u2 = g0.z - cb;
                        const float v0 = bs.y * inv - u0 * mr;
                        const float v1 = bs.z * inv - u1 * mr;
                        const float v2 = bs.w * inv - u2 * mr;
                        const float a0 = g0.w * v0 + g1.x * v1 + g1.y * v2;
                        const float a1 = g1.x * v0 + g1.z * v1 + g1.w * v2;
                        const float a2 = g1.y * v0 + g1.w * v1 + g2.x * v2;
                        const float bk = mr - (a0 * u0 + a1 * u1 + a2 * u2);
                        A[col] = make_float4(a0, a1, a2, bk);
                    }
                }
            }
            kSlot += k1 - k0;
            if (kSlot >= RSA) kSlot -= RSA;
            kNext = k1;
            __syncthreads();
        }
        // window means of a_k, b_k at p: vertical sums over K rows, every K column
        {
            const int ng = (p1 - p0 + 3) >> 2;
            const int rs = Kw;
            if (gV2.tr < gV2.rpp) {
                for (int cc = gV2.tc; cc < Kw; cc += gV2.cpr) {
                    const float4 *A = ABr + cc;
                    float4 *V = Vb + cc;
                    for (int grp = gV2.tr; grp < ng; grp += gV2.rpp) {
                        const int py0 = p0 + 4 * grp, py1 = min(p1, py0 + 4);
                        const int ylo = max(0, py0 - r), yhi = min(H - 1, py0 + r);
                        int sIn = kSlot - (kNext - ylo);
                        if (sIn < 0) sIn += RSA;
                        float4 sm = ring_sum4(A, rs, RSA, sIn, yhi - ylo + 1);
                        V[(py0 - p0) * rs] = sm;
                        int sA = sIn + (yhi - ylo + 1);
                        if (sA >= RSA) sA -= RSA;
                        int sO = sIn;
                        for (int py = py0 + 1; py < py1; ++py) {
                            if (py + r <= H - 1) {
                                sm = add4(sm, A[sA * rs]);
                                sA = ring_next(sA, RSA);
                            }
                            if (py - r - 1 >= 0) {
                                sm = sub4(sm, A[sO * rs]);
                                sO = ring_next(sO, RSA);
                            }
                            V[(py - p0) * rs] = sm;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (gH2.tr < gH2.rpp) {
            for (int chunk = gH2.tc; chunk < nchR; chunk += gH2.cpr) {
                const int px0 = Rx0 + chunk * 4, px1 = min(Rx0 + Rw, px0 + 4);
                const int xlo = max(0, px0 - r), xhi = min(W - 1, px0 + r);
                for (int row = gH2.tr; row < p1 - p0; row += gH2.rpp) {
                    const float4 *V = Vb + row * Kw - Kx0;
                    float4 *B = Bb + row * Rw - Rx0;
                    float4 sm = strided_sum4(V + xlo, 1, xhi - xlo + 1);
                    B[px0] = sm;
                    for (int px = px0 + 1; px < px1; ++px) {
                        if (px + r <= W - 1) sm = add4(sm, V[px + r]);
                        if (px - r - 1 >= 0) sm = sub4(sm, V[px - r - 1]);
                        B[px] = sm;
                    }
                }
            }
        }
        __syncthreads();
        if (gR.tr < gR.rpp) {
            for (int row = gR.tr; row < p1 - p0; row += gR.rpp) {
                const int py = p0 + row;
                const int ny = min(H - 1, py + r) - max(0, py - r) + 1;
                const float4 *B = Bb + row * Rw;
                const size_t rowb = (size_t)py * W;
                for (int col = gR.tc; col < Rw; col += gR.cpr) {
                    const int px = Rx0 + col;
                    const float n = (float)((min(W - 1, px + r) - max(0, px - r) + 1) * ny);
                    const float4 l = load_px(P.L, rowb + px, fmt);
                    const float gu = __fmaf_rn(l.x, inv255, -cr), gv = __fmaf_rn(l.y, inv255, -cg);
                    const float gw = __fmaf_rn(l.z, inv255, -cb);
                    const float4 b4 = B[col];
                    const float phi = __fmaf_rn(b4.x, gu, __fmaf_rn(b4.y, gv, __fmaf_rn(b4.z, gw, b4.w))) / n;
                    out[(size_t)row * pitch + (p0 - Ry0) * (size_t)pitch + col] = phi;
                }
            }
        }
        __syncthreads();
    }
}

// LE-BF data term (Sec. 4): phi_p(f) = sum over the (4r'+1)^2 window of p,
// clipped to the image, of exp(-|I_p - I_s|_1 / gamma) rho(s|f), the weights on
// the 0..255 left colours and not normalised.  rho is computed once per pixel of
// M (the region grown by the window radius) into shared memory, packed with the
// pixel's colours in one 8-byte word; each output pixel then sums its window row
// by row (row partial sums keep the FP32 error of the 1681-term sum near that of
// 82 terms).  A weight is 2^(-d log2(e) / gamma) for the integer L1 distance d
// (byte-wise SAD of the packed colours), on the special-function unit: one
// 8-byte shared load, the SAD, one FMA for the exponent, ex2.approx and the FMA
// of the sum per window pixel.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ void region_unary_bf(const DevPlanes &P, const KParams &kp, int Rx0, int Ry0, int Rw, int Rh, float la,
                                float lb, float lc, float *sm, float *out, int pitch) {
    const int H = P.H, W = P.W, R = 2 * kp.r;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int Mx0 = max(0, Rx0 - R), Mx1 = min(W, Rx0 + Rw + R);
    const int My0 = max(0, Ry0 - R), My1 = min(H, Ry0 + Rh + R);
    const int Mw = Mx1 - Mx0, Mh = My1 - My0;
    float2 *cr = reinterpret_cast<float2 *>(sm);  // [Mh][Mw]: (packed R, G, B bits, rho)
    const int fmt = P.fmt;
    const float oma = 1.0f - kp.alpha_grad;
    float sl;
    const float sh = two_sum(1.0f, -la, sl);
    for (int j = tid; j < Mw * Mh; j += nt) {
        const int my = j / Mw, mx = j - my * Mw;
        const int y = My0 + my, x = Mx0 + mx;
        // warp offset of row y relative to column Mx0, float-float (as region_unary_gf)
        float e1, e2, e3, e4;
        const float p = two_prod(sh, (float)Mx0, e1);
        const float q = two_prod(lb, (float)y, e2);
        const float t1 = two_sum(p, -q, e3);
        const float t2 = two_sum(t1, -lc, e4);
        const float lo = __fadd_rn(__fadd_rn(__fsub_rn(e1, e2), __fadd_rn(e3, e4)), __fmul_rn(sl, (float)Mx0));
        const float th = fminf(fmaxf(t2, -1.0e9f), 1.0e9f);
        const float fl = floorf(th);
        float F = __fadd_rn(__fsub_rn(th, fl), lo);
        int I = (int)fl;
        if (F < 0.f) {
            F += 1.f;
            I -= 1;
        } else if (F >= 1.f) {
            F -= 1.f;
            I += 1;
        }
        const size_t rowb = (size_t)y * W;
        const float4 l = load_px(P.L, rowb + x, fmt);
        const float dx = (float)mx;
        const float g = __fmaf_rn(sh, dx, __fmaf_rn(sl, dx, F));
        const float gf = floorf(g);
        float t = g - gf;
        int i0 = I + (int)gf;
        if (i0 < 0) {
            i0 = 0;
            t = 0.f;
        } else if (i0 >= W - 1) {
            i0 = W - 1;
            t = 0.f;
        }
        const int i1 = min(i0 + 1, W - 1);
        const float4 r0 = load_px(P.R, rowb + i0, fmt), r1 = load_px(P.R, rowb + i1, fmt);
        const float rr = fmaf(t, r1.x - r0.x, r0.x);
        const float rg = fmaf(t, r1.y - r0.y, r0.y);
        const float rb = fmaf(t, r1.z - r0.z, r0.z);
        const float rd = fmaf(t, r1.w - r0.w, r0.w);
        const float cdist = fabsf(l.x - rr) + fabsf(l.y - rg) + fabsf(l.z - rb);
        const float gdist = fabsf(l.w - rd);
        const uint32_t pc = (uint32_t)l.x | ((uint32_t)l.y << 8) | ((uint32_t)l.z << 16);
        cr[j] = make_float2(__uint_as_float(pc), rho_mix(cdist, gdist, kp, oma));
    }
    __syncthreads();
    // exponent of a weight: -k d with k = log2(e) / gamma; d enters as the float
    // 2^23 + d (its bits are 0x4B000000 | d), so one FMA gives -k d exactly rounded
    const float nk = -kp.bf_log2e_inv_gamma, c0 = 8388608.0f * kp.bf_log2e_inv_gamma;
    for (int j = tid; j < Rw * Rh; j += nt) {
        const int ry = j / Rw, rx = j - ry * Rw;
        const int py = Ry0 + ry, px = Rx0 + rx;
        const uint32_t cp = __float_as_uint(cr[(py - My0) * Mw + (px - Mx0)].x);
        const int sx0 = max(0, px - R) - Mx0, sx1 = min(W - 1, px + R) - Mx0;
        float sum = 0.f;
        for (int sy = max(0, py - R); sy <= min(H - 1, py + R); ++sy) {
            const float2 *row = cr + (size_t)(sy - My0) * Mw;
            float rs = 0.f;
            for (int sx = sx0; sx <= sx1; ++sx) {
                const float2 e = row[sx];
                const float d = __uint_as_float(0x4B000000u | __vsadu4(cp, __float_as_uint(e.x)));
                rs = fmaf(ex2_approx(fmaf(d, nk, c0)), e.y, rs);
            }
            sum += rs;
        }
        out[(size_t)ry * pitch + rx] = sum;
    }
    __syncthreads();
}

// data term of one label over one region: guided filter (LE-GF) or bilateral weights (LE-BF)
__device__ __forceinline__ void region_unary(const DevPlanes &P, const KParams &kp, int Rx0, int Ry0, int Rw, int Rh,
                                             float la, float lb, float lc, float *sm, float *out, int pitch) {
    if (kp.bf)
        region_unary_bf(P, kp, Rx0, Ry0, Rw, Rh, la, lb, lc, sm, out, pitch);
    else
        region_unary_gf(P, kp, Rx0, Ry0, Rw, Rh, la, lb, lc, sm, out, pitch);
}

// ---------------------------------------------------------------------------
// A3 + A4 by one warp: the data term of one label over one region whose
// filtering region M is at most 32 NC pixels wide.  Lane l owns the M columns
// l, l + 32, ..., and the warp walks down the rows of M once:
//   * raw cost rho (Eq. photofunc) of the new row and its guide products
//     (I - c) rho enter per-lane vertical window sums; the row that leaves the
//     window is subtracted (its rho from a per-lane ring in shared memory, its
//     products recomputed from the left image);
//   * each completed row of K (R grown by r') gets its horizontal window sums
//     from an inclusive prefix sum across the lanes (warp shuffles), then the
//     guided-filter coefficients a_k, b_k (Eq. gf);
//   * a_k, b_k enter a second pair of vertical window sums (their ring is in
//     shared memory too), and each completed row of R gets the horizontal
//     window sums of the coefficients the same way and phi_p = mean(a) . I_p +
//     mean(b).
// Every window sum is exact: the raw-cost channels are summed as 32-bit
// fixed-point integers (scale kp.q1, a power of two chosen so that no window sum
// of (2r'+1)^2 terms can overflow; prefix sums wrap modulo 2^32, which leaves
// each difference exact), the coefficients as 64-bit fixed-point integers
// (scale kp.q2, sums mod 2^64).  So the result depends on no summation order, launch shape or
// strip size, and the only rounding in the sums is that of each term to its
// fixed-point grid (2^-21 for the default raw costs, 2^-33 for coefficients).
// ring: shared memory owned by the warp (warp_ring_floats).  The next M row's
// image values are loaded while a row is processed.
// ---------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

template <typename T, int NC>
__device__ __forceinline__ void warp_prefix(T (&p)[NC], int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            const T t = __shfl_up_sync(kFull, p[j], o);
            if (lane >= o) p[j] += t;
        }
    }
    T carry = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        p[j] += carry;
        carry = __shfl_sync(kFull, p[j], 31);
    }
}
// element m (0 <= m < 32 NC) of a prefix array held as p[m >> 5] on lane m & 31;
// m < 0 gives 0.  Every lane of the warp must call it.
template <typename T, int NC>
__device__ __forceinline__ T warp_at(const T (&p)[NC], int m) {
    const int src = m & 31, blk = m >> 5;
    T v = 0;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const T t = __shfl_sync(kFull, p[j], src);
        if (j == blk) v = t;
    }
    return m < 0 ? (T)0 : v;
}

__device__ __forceinline__ int yEndOf(int Ry0, int Rh, int r) { return Ry0 + Rh + 2 * r; }

// image values of one M pixel that its raw cost needs: the left pixel, the two
// right pixels of the linear tap and its weight, and the left pixel of the row
// leaving the vertical window
struct RowPx {
    float4 l, r0, r1, ll;
    float t;
};

template <int NC>
__device__ __forceinline__ void fetch_row(const DevPlanes &P, int y, int yl, bool add, bool leave, int Mx0, int Mx1,
                                          int Rx0, float sh, float sl, float lb, float lc, int lane,
                                          RowPx (&o)[NC]) {
    const int W = P.W, fmt = P.fmt;
    int Ib = 0;
    float Fb = 0.f;
    if (add) row_offset(sh, sl, lb, lc, Rx0, y, Ib, Fb);
    const size_t rowb = (size_t)y * W, rowl = (size_t)yl * W;
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const int x = Mx0 + lane + 32 * j;
        if (x >= Mx1) continue;
        if (add) {
            o[j].l = load_px(P.L, rowb + x, fmt);
            const float dx = (float)(x - Rx0);
            const float g = __fmaf_rn(sh, dx, __fmaf_rn(sl, dx, Fb));
            const float gf = floorf(g);
            float t = g - gf;
            int i0 = Ib + (int)gf;
            if (i0 < 0) {
                i0 = 0;
                t = 0.f;
            } else if (i0 >= W - 1) {
                i0 = W - 1;
                t = 0.f;
            }
            o[j].t = t;
            o[j].r0 = load_px(P.R, rowb + i0, fmt);
            o[j].r1 = load_px(P.R, rowb + min(i0 + 1, W - 1), fmt);
        }
        if (leave) o[j].ll = load_px(P.L, rowl + x, fmt);
    }
}

// raw cost (Eq. photofunc) from the fetched image values (the steps of raw_cost)
__device__ __forceinline__ float rho_of(const RowPx &q, const KParams &kp, float oma) {
    const float rr = fmaf(q.t, q.r1.x - q.r0.x, q.r0.x);
    const float rg = fmaf(q.t, q.r1.y - q.r0.y, q.r0.y);
    const float rb = fmaf(q.t, q.r1.z - q.r0.z, q.r0.z);
    const float rd = fmaf(q.t, q.r1.w - q.r0.w, q.r0.w);
    const float col = fabsf(q.l.x - rr) + fabsf(q.l.y - rg) + fabsf(q.l.z - rb);
    const float gd = fabsf(q.l.w - rd);
    return rho_mix(col, gd, kp, oma);
}

// ring (shared memory of the calling warp): raw costs [2r'+1][mwp], then the
// guided-filter coefficients [2r'+1][4][kwp]; mwp, kwp >= the widths of M and K
template <int NC>
__device__ void warp_unary_gf(const DevPlanes &P, const KParams &kp, int Rx0, int Ry0, int Rw, int Rh, float la,
                              float lb, float lc, float *ring, int mwp, int kwp, float *out, int pitch) {
    const int H = P.H, W = P.W, r = kp.r, fmt = P.fmt;
    const int lane = threadIdx.x & 31;
    const int Mx0 = max(0, Rx0 - 2 * r), Mx1 = min(W, Rx0 + Rw + 2 * r);
    const int My0 = max(0, Ry0 - 2 * r), My1 = min(H, Ry0 + Rh + 2 * r);
    const int Kx0 = max(0, Rx0 - r), Kx1 = min(W, Rx0 + Rw + r);
    const int Ky0 = max(0, Ry0 - r), Ky1 = min(H, Ry0 + Rh + r);
    const int Kw = Kx1 - Kx0;
    const int WIN = 2 * r + 1;
    float *rho_ring = ring;                 // [WIN][mwp]
    float *ab_ring = ring + WIN * mwp;      // [WIN][4][kwp]
    const float4 cen4 = load_px(P.L, (size_t)(Ry0 + Rh / 2) * W + (Rx0 + Rw / 2), fmt);
    const float inv255 = 1.0f / 255.0f;
    const float cr = cen4.x * inv255, cg = cen4.y * inv255, cb = cen4.z * inv255;
    float sl;
    const float sh = two_sum(1.0f, -la, sl);
    const float oma = 1.0f - kp.alpha_grad;
    const float q1 = kp.q1, q2 = kp.q2;

    unsigned vs[4][NC];            // vertical window sums of the raw-cost channels (fixed point, mod 2^32)
    unsigned long long va[4][NC];  // vertical window sums of a_k (3) and b_k (fixed point, mod 2^64)
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < NC; ++j) {
            vs[c][j] = 0u;
            va[c][j] = 0ull;
        }
    const int yS1 = min(yEndOf(Ry0, Rh, r), Ky1 + r);  // rows that feed stage 1
    const int yEnd = yEndOf(Ry0, Rh, r);               // one past the last row that completes an R row
    RowPx cur[NC], nxt[NC];
    fetch_row<NC>(P, My0, My0 - WIN, My0 < My1, false, Mx0, Mx1, Rx0, sh, sl, lb, lc, lane, cur);
    int slot1 = 0, slot2 = 0;  // ring slots of the row entering stage 1 / K row entering stage 2
    for (int y = My0; y < yEnd; ++y) {
        // the next row's image values are loaded while this row is processed
        if (y + 1 < yS1)
            fetch_row<NC>(P, y + 1, y + 1 - WIN, y + 1 < My1, y + 1 - WIN >= My0, Mx0, Mx1, Rx0, sh, sl, lb, lc,
                          lane, nxt);
        // ---- stage 1: raw-cost channels of M row y; K row ky = y - r completes
        if (y < yS1) {
            const bool add = y < My1, leave = y - WIN >= My0;
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const int c = lane + 32 * j;
                if (Mx0 + c >= Mx1) continue;
                float *slotp = rho_ring + slot1 * mwp + c;  // the leaving row's slot is the entering row's
                if (leave) {
                    const float rho = *slotp;
                    const float4 l = cur[j].ll;
                    vs[0][j] -= (unsigned)__float2int_rn(__fmul_rn(rho, q1));
                    vs[1][j] -= (unsigned)__float2int_rn(__fmul_rn(__fmul_rn(__fmaf_rn(l.x, inv255, -cr), rho), q1));
                    vs[2][j] -= (unsigned)__float2int_rn(__fmul_rn(__fmul_rn(__fmaf_rn(l.y, inv255, -cg), rho), q1));
                    vs[3][j] -= (unsigned)__float2int_rn(__fmul_rn(__fmul_rn(__fmaf_rn(l.z, inv255, -cb), rho), q1));
                }
                if (add) {
                    const float4 l = cur[j].l;
                    const float rho = rho_of(cur[j], kp, oma);
                    *slotp = rho;
                    vs[0][j] += (unsigned)__float2int_rn(__fmul_rn(rho, q1));
                    vs[1][j] += (unsigned)__float2int_rn(__fmul_rn(__fmul_rn(__fmaf_rn(l.x, inv255, -cr), rho), q1));
                    vs[2][j] += (unsigned)__float2int_rn(__fmul_rn(__fmul_rn(__fmaf_rn(l.y, inv255, -cg), rho), q1));
                    vs[3][j] += (unsigned)__float2int_rn(__fmul_rn(__fmul_rn(__fmaf_rn(l.z, inv255, -cb), rho), q1));
                }
            }
            if (++slot1 == WIN) slot1 = 0;
#pragma unroll
            for (int j = 0; j < NC; ++j) cur[j] = nxt[j];
        }
        const int ky = y - r;
        if (ky < Ky0) continue;
        // ---- stage 2: coefficients of K row ky (when it is a row of K) enter the
        // vertical sums; the K row ky - WIN leaves
        {
            const int kyl = ky - WIN;
            const bool real = ky < Ky1;
            float a[4][NC];
            if (real) {
                const int ny = min(H - 1, ky + r) - max(0, ky - r) + 1;
                unsigned p[4][NC];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
#pragma unroll
                    for (int j = 0; j < NC; ++j) p[c][j] = vs[c][j];
                    warp_prefix<unsigned, NC>(p[c], lane);
                }
#pragma unroll
                for (int j = 0; j < NC; ++j) {
                    a[0][j] = a[1][j] = a[2][j] = a[3][j] = 0.f;
                    if (32 * j >= Kw) continue;  // (warp-uniform) no K column in this block
                    const int kx = Kx0 + lane + 32 * j;
                    const int hi = min(W - 1, kx + r) - Mx0, lo = max(0, kx - r) - Mx0 - 1;
                    float S[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        S[c] = (float)(int)(warp_at<unsigned, NC>(p[c], hi) - warp_at<unsigned, NC>(p[c], lo));
                    if (kx < Kx1) {
                        const int nx = min(W - 1, kx + r) - max(0, kx - r) + 1;
                        const float inv = 1.0f / __fmul_rn((float)(nx * ny), q1);
                        const float mr = __fmul_rn(S[0], inv);
                        const float4 *G = P.gst + 3 * ((size_t)ky * W + kx);
                        const float4 g0 = G[0], g1 = G[1], g2 = G[2];
                        const float u0 = g0.x - cr, u1 = g0.y - cg, u2 = g0.z - cb;
                        const float v0 = __fmaf_rn(-u0, mr, __fmul_rn(S[1], inv));
                        const float v1 = __fmaf_rn(-u1, mr, __fmul_rn(S[2], inv));
                        const float v2 = __fmaf_rn(-u2, mr, __fmul_rn(S[3], inv));
                        const float a0 = __fmaf_rn(g0.w, v0, __fmaf_rn(g1.x, v1, __fmul_rn(g1.y, v2)));
                        const float a1 = __fmaf_rn(g1.x, v0, __fmaf_rn(g1.z, v1, __fmul_rn(g1.w, v2)));
                        const float a2 = __fmaf_rn(g1.y, v0, __fmaf_rn(g1.w, v1, __fmul_rn(g2.x, v2)));
                        a[0][j] = a0;
                        a[1][j] = a1;
                        a[2][j] = a2;
                        a[3][j] = __fsub_rn(mr, __fmaf_rn(a0, u0, __fmaf_rn(a1, u1, __fmul_rn(a2, u2))));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                const int c = lane + 32 * j;
                if (Kx0 + c >= Kx1) continue;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    float *slotp = ab_ring + (slot2 * 4 + ch) * kwp + c;
                    if (kyl >= Ky0) va[ch][j] -= (unsigned long long)__float2ll_rn(__fmul_rn(*slotp, q2));
                    if (real) {
                        *slotp = a[ch][j];
                        va[ch][j] += (unsigned long long)__float2ll_rn(__fmul_rn(a[ch][j], q2));
                    }
                }
            }
            if (++slot2 == WIN) slot2 = 0;
        }
        // ---- R row py = ky - r completes: horizontal sums of the coefficients, phi
        const int py = ky - r;
        if (py < Ry0) continue;
        {
            const int ny = min(H - 1, py + r) - max(0, py - r) + 1;
            unsigned long long p[4][NC];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
#pragma unroll
                for (int j = 0; j < NC; ++j) p[c][j] = va[c][j];
                warp_prefix<unsigned long long, NC>(p[c], lane);
            }
            const size_t rowb = (size_t)py * W;
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                if (32 * j >= Rw) continue;  // (warp-uniform) no R column in this block
                const int px = Rx0 + lane + 32 * j;
                const int hi = min(W - 1, px + r) - Kx0, lo = max(0, px - r) - Kx0 - 1;
                float S[4];
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    S[c] = __ll2float_rn((long long)(warp_at<unsigned long long, NC>(p[c], hi) -
                                                     warp_at<unsigned long long, NC>(p[c], lo)));
                if (px < Rx0 + Rw) {
                    const int nx = min(W - 1, px + r) - max(0, px - r) + 1;
                    const float4 l = load_px(P.L, rowb + px, fmt);
                    const float gu = __fmaf_rn(l.x, inv255, -cr), gv = __fmaf_rn(l.y, inv255, -cg);
                    const float gw = __fmaf_rn(l.z, inv255, -cb);
                    const float num = __fmaf_rn(S[0], gu, __fmaf_rn(S[1], gv, __fmaf_rn(S[2], gw, S[3])));
                    out[(size_t)(py - Ry0) * pitch + (px - Rx0)] = __fdiv_rn(num, __fmul_rn((float)(nx * ny), q2));
                }
            }
        }
    }
}

// shared-memory floats of one warp's rings for M and K at most mwp and kwp wide
__host__ __device__ inline int warp_ring_floats(int r, int mwp, int kwp) { return (2 * r + 1) * (mwp + 4 * kwp); }



// ---------------------------------------------------------------------------
// A5: expansion-move graph of one node
// ---------------------------------------------------------------------------
struct NodeCaps {
    int cap_s, cap_t;  // s->p (taken when x_p = 1), p->t (taken when x_p = 0)
    int k[4];          // p -> forward neighbour inside R
    long long cst;     // constant: lowered A's of the forward pairs + min(U0, U1)
    int nclamp;
};

// Node p = (x0+ix, y0+iy) of region [x0,x0+w) x [y0,y0+h); al = candidate,
// phi_al = phi_p(alpha); lab holds the current labels and cost cache.
__device__ void build_node(const DevPlanes &P, const KParams &kp, const float4 *lab, const float4 &al,
                           float phi_al, int x0, int y0, int w, int h, int ix, int iy, NodeCaps &o) {
    const int H = P.H, W = P.W;
    const int pu = x0 + ix, pv = y0 + iy;
    const float fu = (float)pu, fv = (float)pv;
    const float4 fp = lab[(size_t)pv * W + pu];
    int U0 = q_cost(fp.w, kp.S), U1 = q_cost(phi_al, kp.S);
    long long cst = 0;
    int ncl = 0;
    const float4 wp = P.wfw[(size_t)pv * W + pu];
    // the eight neighbours' labels, loaded together before any is used (coordinates
    // clamped to the image; a direction that leaves the image is skipped below)
    float4 fqa[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int qu = min(max(pu + dir_dx(k), 0), W - 1), qv = min(max(pv + dir_dy(k), 0), H - 1);
        fqa[k] = lab[(size_t)qv * W + qu];
    }
    // psi(f_p, alpha) on every pair of p: its coefficient differences and its value
    // at p are shared by the 8 neighbours (the term of a backward pair (q, p) with
    // alpha at q is psi(f_p, alpha) on the same pair: each label is evaluated at
    // both ends, and the differences are antisymmetric bit for bit)
    const DDCoef dpa = dd_coef(fp, al);
    const float dpa_p = dd_eval(dpa, fu, fv);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int d = k & 3;
        const bool fwd = k < 4;
        if (fwd) o.k[d] = 0;
        const int qu = pu + dir_dx(k), qv = pv + dir_dy(k);
        if (qu < 0 || qu >= W || qv < 0 || qv >= H) continue;
        const float gu = (float)qu, gv = (float)qv;
        const float wl = fwd ? comp(wp, d) : comp(P.wfw[(size_t)qv * W + qu], d);
        const bool qin = qu >= x0 && qu < x0 + w && qv >= y0 && qv < y0 + h;
        if (!qin) {
            const float4 fq = fqa[k];
            const DDCoef dpq = dd_coef(fp, fq), daq = dd_coef(al, fq);
            U0 += q_of(wl, kp.tau_dis, kp.S, dd_eval(dpq, fu, fv), dd_eval(dpq, gu, gv));
            U1 += q_of(wl, kp.tau_dis, kp.S, dd_eval(daq, fu, fv), dd_eval(daq, gu, gv));
        } else if (fwd) {
            const float4 fq = fqa[k];
            const DDCoef dpq = dd_coef(fp, fq), daq = dd_coef(al, fq);
            int A = q_of(wl, kp.tau_dis, kp.S, dd_eval(dpq, fu, fv), dd_eval(dpq, gu, gv));
            const int B = q_of(wl, kp.tau_dis, kp.S, dpa_p, dd_eval(dpa, gu, gv));
            const int C = q_of(wl, kp.tau_dis, kp.S, dd_eval(daq, fu, fv), dd_eval(daq, gu, gv));
            if (A > B + C) {
                A = B + C;
                ++ncl;
            }
            cst += A;
            U1 += C - A;
            o.k[d] = B + C - A;
        } else {
            // backward neighbour q: the pair (q, p) is forward from q, whose C
            // term psi(alpha at q, f_p at p) lands on p's unary with a minus sign
            U1 -= q_of(wl, kp.tau_dis, kp.S, dd_eval(dpa, gu, gv), dpa_p);
        }
    }
    const int m = min(U0, U1);
    o.cap_s = U1 - m;
    o.cap_t = U0 - m;
    o.cst = cst + m;
    o.nclamp = ncl;
}

// block-wide sum of a long long (all threads get the result)
__device__ long long block_sum_ll(long long v, long long *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int i = 0; i < nw; ++i) s += red[i];
        red[32] = s;
    }
    __syncthreads();
    return red[32];
}

// ---------------------------------------------------------------------------
// A6: CTA push-relabel on a w x h grid region held in shared memory
//   res[k*n + i] : residual capacity of i -> neighbour k (8 directions)
//   v[i]         : excess minus residual sink capacity (excess = max(v,0),
//                  residual p->t = max(-v,0)); excess reaching a node with
//                  residual sink capacity is pushed to the sink at once
//   hh[i]        : height (kInf = cannot reach the sink)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dir_off(int k, int w) { return dir_dx(k) + dir_dy(k) * w; }

// Row and column of the indices j0, j0 + step, j0 + 2 step, ... of a row-major
// grid with rows of w entries, advanced by exact integer steps (one division
// at construction, none per index).
struct RowCol {
    int y, x, dy, dx, w;
    __device__ RowCol(int j0, int step, int w_) : w(w_) {
        y = j0 / w;
        x = j0 - y * w;
        dy = step / w;
        dx = step - dy * w;
    }
    __device__ __forceinline__ void next() {
        y += dy;
        x += dx;
        if (x >= w) {
            x -= w;
            ++y;
        }
    }
};

// Exact distances to the sink in the residual graph, by a bit-parallel BFS
// backwards from the nodes with residual sink capacity.  Rows of the region
// are bit strings of WPR 32-bit words; for each direction k a bitplane marks
// the nodes with residual capacity toward neighbour k.  One BFS level is, per
// word, the OR over k of (plane_k AND frontier shifted by the offset of k),
// minus the visited set.  Returns whether some node with excess can still
// reach the sink; *levels gets the BFS depth.
//   bits: 8 planes + 2 frontiers + visited, each h * WPR words
__device__ bool global_relabel(int n, int w, int h, const int *res, const int *v, uint16_t *hh, uint32_t *bits,
                               int *levels) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    const int WPR = (w + 31) >> 5, NW = h * WPR;
    uint32_t *M = bits, *Fa = bits + 8 * NW, *Fb = Fa + NW, *VIS = Fb + NW;
    // planes and seeds: one warp per row, one pass per row word, lane = bit
    for (int y = warp; y < h; y += nwarp) {
        for (int wi = 0; wi < WPR; ++wi) {
            const int word = y * WPR + wi;
            const int x = wi * 32 + lane;
            const bool in = x < w;
            const int i = y * w + x;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                bool pred = false;
                if (in) pred = res[k * n + i] > 0;
                const uint32_t m = __ballot_sync(0xffffffffu, pred);
                if (lane == 0) M[k * NW + word] = m;
            }
            bool seed = false;
            if (in) seed = v[i] < 0;
            const uint32_t m = __ballot_sync(0xffffffffu, seed);
            if (lane == 0) {
                Fa[word] = m;
                VIS[word] = m;
            }
            if (in) hh[i] = seed ? 1 : kInf;
        }
    }
    __syncthreads();
    uint32_t *Fc = Fa, *Fn = Fb;
    int level = 1;
    for (;;) {
        int any = 0;
        RowCol rw(tid, nt, WPR);
        for (int word = tid; word < NW; word += nt, rw.next()) {
            const int y = rw.y, wi = rw.x;
            const uint32_t vis = VIS[word];
            uint32_t cand = 0;
            {
                // frontier words of rows y-1, y, y+1 around column word wi, shifted by
                // dx = -1, 0, +1: sh[dy+1][dx+1] holds, at bit b, the frontier bit of
                // node (x + dx, y + dy) for the node x at bit b.  Every load is issued
                // at once, at indices clamped to the grid; words outside it count as 0.
                uint32_t sh[3][3], pl[8];
                const int wl = max(wi - 1, 0), wr = min(wi + 1, WPR - 1);
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int yy = y + r - 1;
                    const bool rin = yy >= 0 && yy < h;
                    const uint32_t *F = Fc + min(max(yy, 0), h - 1) * WPR;
                    uint32_t c = F[wi], lw = F[wl], rw2 = F[wr];
                    if (!rin) c = lw = rw2 = 0u;
                    if (wi == 0) lw = 0u;
                    if (wi + 1 >= WPR) rw2 = 0u;
                    sh[r][0] = (c << 1) | (lw >> 31);  // dx = -1
                    sh[r][1] = c;                       // dx = 0
                    sh[r][2] = (c >> 1) | (rw2 << 31);  // dx = +1
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) pl[k] = M[k * NW + word];
#pragma unroll
                for (int k = 0; k < 8; ++k) cand |= pl[k] & sh[dir_dy(k) + 1][dir_dx(k) + 1];
                // only bits of nodes inside the row can be reached
                const int tail = w - wi * 32;
                cand &= ~vis & (tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u));
            }
            Fn[word] = cand;
            if (cand) {
                VIS[word] = vis | cand;
                any = 1;
                uint32_t c = cand;
                const int base = y * w + wi * 32;
                while (c) {
                    const int b = __ffs(c) - 1;
                    c &= c - 1;
                    hh[base + b] = (uint16_t)(level + 1);
                }
            }
        }
        if (!__syncthreads_or(any)) break;
        uint32_t *t = Fc;
        Fc = Fn;
        Fn = t;
        ++level;
    }
    *levels += level;
    int act = 0;
    for (int i = tid; i < n; i += nt) act |= (v[i] > 0 && hh[i] != kInf);
    return __syncthreads_or(act) != 0;
}

// The same as a separate function: kernels of up to 256 threads call it, so
// that its code does not take part in their register allocation.
__device__ __noinline__ bool global_relabel_outlined(int n, int w, int h, const int *res, const int *v, uint16_t *hh,
                                                     uint32_t *bits, int *levels) {
    return global_relabel(n, w, h, res, v, hh, bits, levels);
}

// Terminal reduction before the max-flow: a node's excess beyond what its
// outgoing n-links can carry can never leave it, and a node's sink capacity
// beyond what its incoming n-links can bring is never used.  Clamping
// v = cap_s - cap_t to [-(in + 1), out + 1] keeps the max-flow value and the
// minimal sink side unchanged: a node with cap_s > out lies on the source side
// of every minimum cut and one with cap_t > in on the sink side, and the slack
// of one unit keeps these strict.  Needs res (initial capacities) and v.
__device__ void clamp_terminals(int n, int w, int h, const int *res, int *v) {
    RowCol rc(threadIdx.x, blockDim.x, w);
    for (int i = threadIdx.x; i < n; i += blockDim.x, rc.next()) {
        const int e = v[i];
        if (e > 0) {
            int out = 1;
#pragma unroll
            for (int k = 0; k < 8; ++k) out += res[k * n + i];
            v[i] = min(e, out);
        } else if (e < 0) {
            const int iy = rc.y, ix = rc.x;
            int in = 1;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int jx = ix + dir_dx(k), jy = iy + dir_dy(k);
                if (jx < 0 || jx >= w || jy < 0 || jy >= h) continue;
                // the edge from neighbour j back to i runs in direction k^4 at j
                in += res[(k ^ 4) * n + i + dir_off(k, w)];
            }
            v[i] = max(e, -in);
        }
    }
}

// Global relabel of a region of at most 32 x 32 nodes (called by every thread of
// the CTA): the warps build the residual bitplanes and the BFS seeds one row each
// (lane = column) into shared memory; warp 0 then keeps row y's planes and BFS
// words in lane y and moves frontier rows between lanes with shuffles, so no BFS
// level needs a CTA barrier; every thread then checks its nodes for excess that
// can reach the sink.  Same result as global_relabel: exact distances to the sink
// in hh (kInf where the sink cannot be reached).
//   bits: 9 h words (8 planes and the seeds, row-indexed)
__device__ __noinline__ bool small_relabel(int n, int w, int h, const int *res, const int *v, uint16_t *hh,
                                           uint32_t *bits, int *levels) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
    const uint32_t full = 0xffffffffu;
    for (int y = warp; y < h; y += nwarp) {
        const bool in = lane < w;
        const int i = y * w + lane;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            bool p = false;
            if (in) p = res[k * n + i] > 0;
            const uint32_t m = __ballot_sync(full, p);
            if (lane == 0) bits[k * h + y] = m;
        }
        bool seed = false;
        if (in) seed = v[i] < 0;
        const uint32_t m = __ballot_sync(full, seed);
        if (lane == 0) bits[8 * h + y] = m;
        if (in) hh[i] = seed ? 1 : kInf;
    }
    __syncthreads();
    if (warp == 0) {
        const uint32_t rowmask = w >= 32 ? full : ((1u << w) - 1u);
        uint32_t M[8], F = 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) M[k] = lane < h ? bits[k * h + lane] : 0u;
        if (lane < h) F = bits[8 * h + lane];
        uint32_t VIS = F;
        int level = 1;
        for (;;) {
            const uint32_t up = __shfl_up_sync(full, F, 1), dn = __shfl_down_sync(full, F, 1);
            const uint32_t rows[3] = {lane > 0 ? up : 0u, F, lane + 1 < h ? dn : 0u};  // dy = -1, 0, +1
            uint32_t cand = 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint32_t r = rows[dir_dy(k) + 1];
                const int dx = dir_dx(k);
                cand |= M[k] & (dx > 0 ? (r >> 1) : (dx < 0 ? (r << 1) : r));
            }
            cand &= ~VIS & rowmask;
            if (lane >= h) cand = 0u;
            VIS |= cand;
            F = cand;
            uint32_t c = cand;
            while (c) {
                const int b = __ffs(c) - 1;
                c &= c - 1;
                hh[lane * w + b] = (uint16_t)(level + 1);
            }
            if (!__any_sync(full, cand != 0u)) break;
            ++level;
        }
        *levels += level;
    }
    __syncthreads();
    int act = 0;
    for (int i = tid; i < n; i += blockDim.x) act |= (v[i] > 0 && hh[i] != kInf);
    return __syncthreads_or(act) != 0;
}

struct CutCount {
    int rounds, relabels, levels;
};

// One push of node i with e > 0 excess at height hu: along admissible edges (to
// a neighbour one level lower) as far as the residual capacities allow, then,
// with excess left and no admissible edge, a relabel from the heights read here.
// All loads come first and are independent: the eight neighbour heights are read
// together with the residuals, at indices clamped to the region (a direction
// that leaves the region has no residual capacity, so what is read there is
// never used).  The pushes are decided in registers, and
// the updates are fire-and-forget shared atomics (a neighbour may push into i's
// reverse edges or excess at the same time; it only ever adds).  A stale
// height read only costs extra rounds: the global relabel restores exact
// heights and decides termination.
__device__ __forceinline__ void push_node(int n, int w, int *res, int *v, uint16_t *hh, int i, int e, int hu) {
    int r[8], hn[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = res[k * n + i];
#pragma unroll
    for (int k = 0; k < 8; ++k) hn[k] = (int)hh[min(max(i + dir_off(k, w), 0), n - 1)];
#pragma unroll
    for (int k = 0; k < 8; ++k) hn[k] = r[k] > 0 ? hn[k] : (int)kInf;
    int left = e, mh = kInf;
    int d[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        d[k] = 0;
        if (r[k] > 0 && hn[k] + 1 == hu && left > 0) {
            d[k] = min(left, r[k]);
            left -= d[k];
        }
        if (r[k] - d[k] > 0) mh = min(mh, hn[k]);
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        if (d[k] == 0) continue;
        const int j = i + dir_off(k, w);
        atomicSub(&res[k * n + i], d[k]);
        atomicAdd(&res[(k ^ 4) * n + j], d[k]);
        atomicAdd(&v[j], d[k]);
    }
    if (left != e) atomicSub(&v[i], e - left);
    if (left > 0) hh[i] = (mh >= n + 1) ? kInf : (uint16_t)(mh + 1);
}

// Maximum preflow.  On return (LEM_OK) hh[i] != kInf exactly for the nodes that
// reach the sink in the residual graph: the minimal sink side of the cut.
// Regions of at most two nodes per thread: each thread pushes its own active
// nodes every round, and one barrier (which also reduces "any node was active")
// ends the round.  Larger regions first compact the active nodes (excess,
// finite height) into a list each round, so warps only run the push path for
// nodes that have work.
//   list: n 16-bit entries; shares storage with the relabel's bitplanes
template <bool kOutline = false>
__device__ int cta_maxflow(int n, int w, int h, int *res, int *v, uint16_t *hh, uint32_t *bits, int max_rounds,
                           int gr_interval, CutCount &cc) {
    // active-node counters of even and odd rounds: a round zeroes the other one, so
    // no barrier is needed to reset the counter at the start of a round
    __shared__ int s_cnt2[2];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    uint16_t *list = (uint16_t *)bits;
    // regions of at most 32 x 32 nodes: the BFS levels of the relabel run on warp 0
    const bool small = w <= 32 && h <= 32;
    auto relabel = [&]() -> bool {
        if (!small)
            return kOutline ? global_relabel_outlined(n, w, h, res, v, hh, bits, &cc.levels)
                            : global_relabel(n, w, h, res, v, hh, bits, &cc.levels);
        return small_relabel(n, w, h, res, v, hh, bits, &cc.levels);
    };
    if (tid == 0) s_cnt2[0] = 0;
    bool act = relabel();
    ++cc.relabels;
    int rounds = 0;
    if (n <= 2 * nt) {
        while (act) {
            if (rounds >= max_rounds) {
                cc.rounds += rounds;
                return LEM_ERR_MAXFLOW_LIMIT;
            }
            int any = 0;
            for (int i = tid; i < n; i += nt) {
                const int e = v[i];
                const int hu = hh[i];
                if (e > 0 && hu != kInf) {
                    any = 1;
                    push_node(n, w, res, v, hh, i, e, hu);
                }
            }
            ++rounds;
            // a round with no active node, or the periodic point, hands over to an
            // exact global relabel (which also decides termination)
            if (!__syncthreads_or(any) || rounds % gr_interval == 0) {
                act = relabel();
                ++cc.relabels;
            }
        }
        cc.rounds += rounds;
        return LEM_OK;
    }
    while (act) {
        if (rounds >= max_rounds) {
            cc.rounds += rounds;
            return LEM_ERR_MAXFLOW_LIMIT;
        }
        int *s_cnt = s_cnt2 + (rounds & 1);
        // four consecutive nodes per thread (one 16-byte load of v, one 8-byte
        // load of hh); a warp appends its active nodes with one atomic, placed by
        // four ballots (list order within a warp: first nodes, then second, ...)
        for (int base = 0; base < n; base += 4 * nt) {
            const int i0 = base + 4 * tid;
            bool a0 = false, a1 = false, a2 = false, a3 = false;
            if (i0 + 3 < n) {
                const int4 vv = *reinterpret_cast<const int4 *>(v + i0);
                const ushort4 h4 = *reinterpret_cast<const ushort4 *>(hh + i0);
                a0 = vv.x > 0 && h4.x != kInf;
                a1 = vv.y > 0 && h4.y != kInf;
                a2 = vv.z > 0 && h4.z != kInf;
                a3 = vv.w > 0 && h4.w != kInf;
            } else if (i0 < n) {
                a0 = v[i0] > 0 && hh[i0] != kInf;
                a1 = i0 + 1 < n && v[i0 + 1] > 0 && hh[i0 + 1] != kInf;
                a2 = i0 + 2 < n && v[i0 + 2] > 0 && hh[i0 + 2] != kInf;
            }
            const uint32_t m0 = __ballot_sync(0xffffffffu, a0), m1 = __ballot_sync(0xffffffffu, a1);
            const uint32_t m2 = __ballot_sync(0xffffffffu, a2), m3 = __ballot_sync(0xffffffffu, a3);
            const int c0 = __popc(m0), c1 = __popc(m1), c2 = __popc(m2), c3 = __popc(m3);
            const int tot = c0 + c1 + c2 + c3;
            if (tot == 0) continue;
            int pos = 0;
            if (lane == 0) pos = atomicAdd(s_cnt, tot);
            pos = __shfl_sync(0xffffffffu, pos, 0);
            const uint32_t lt = (1u << lane) - 1u;
            if (a0) list[pos + __popc(m0 & lt)] = (uint16_t)i0;
            pos += c0;
            if (a1) list[pos + __popc(m1 & lt)] = (uint16_t)(i0 + 1);
            pos += c1;
            if (a2) list[pos + __popc(m2 & lt)] = (uint16_t)(i0 + 2);
            pos += c2;
            if (a3) list[pos + __popc(m3 & lt)] = (uint16_t)(i0 + 3);
        }
        __syncthreads();
        const int cnt = *s_cnt;
        // the other counter is free until the next round's compaction (after the
        // barrier that ends this round)
        if (tid == 0) s_cnt2[(rounds & 1) ^ 1] = 0;
        for (int q = tid; q < cnt; q += nt) {
            const int i = list[q];
            push_node(n, w, res, v, hh, i, v[i], hh[i]);
        }
        ++rounds;
        __syncthreads();
        // a round with no active node, or the periodic point, hands over to an
        // exact global relabel (which also decides termination)
        if (cnt == 0 || rounds % gr_interval == 0) {
            act = relabel();
            ++cc.relabels;
        }
    }
    cc.rounds += rounds;
    return LEM_OK;
}

// shared-memory layout of the CTA min-cut for a w x h region (n = w h nodes)
struct CutSmem {
    int *res;
    int *v;
    uint16_t *hh;
    uint32_t *bits;
};
__device__ __forceinline__ CutSmem cut_layout(void *base, int n) {
    CutSmem c;
    c.res = (int *)base;
    c.v = c.res + 8 * n;
    // heights start on a 16-byte boundary so four of them load as one 8-byte word
    c.hh = (uint16_t *)((char *)base + ((36 * (size_t)n + 15) & ~(size_t)15));
    c.bits = (uint32_t *)(c.hh + ((n + 1) & ~1));
    return c;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// phi_p(f_p) for every pixel, one CTA per pixel (1x1 region)
__global__ void k_pixel_costs(DevPlanes P, KParams kp, float4 *lab) {
    extern __shared__ __align__(16) float smf[];
    const int p = blockIdx.x;
    const int x = p % P.W, y = p / P.W;
    const float4 f = lab[p];
    region_unary(P, kp, x, y, 1, 1, f.x, f.y, f.z, smf, &lab[p].w, 1);
}

// the planes of pair pd (the batch's arrays offset to its pixels)
__device__ __forceinline__ void pair_planes(DevPlanes &P, KParams &kp, const PairDesc &pd) {
    P.H = pd.H;
    P.W = pd.W;
    P.L = px_offset(P.L, pd.off, P.fmt);
    P.R = px_offset(P.R, pd.off, P.fmt);
    P.gst += 3 * pd.off;
    P.wfw += pd.off;
    kp.seed = pd.seed;
    kp.disp_min = pd.disp_min;
    kp.disp_max = pd.disp_max;
}

// P: base planes of all pairs; region i belongs to pair img[i]
__global__ void k_unary_batch(DevPlanes P, KParams kp, const PairDesc *pairs, const int *img, const int4 *regions,
                              const int64_t *offsets, int K, const float *labels, float *costs) {
    extern __shared__ __align__(16) float smf[];
    const int i = blockIdx.x / K, k = blockIdx.x % K;
    pair_planes(P, kp, pairs[img[i]]);
    const int4 R = regions[i];
    const float *l = labels + ((size_t)i * K + k) * 3;
    float *out = costs + offsets[i] + (int64_t)k * R.z * R.w;
    region_unary(P, kp, R.x, R.y, R.z, R.w, l[0], l[1], l[2], smf, out, R.z);
}

// P, lab_all: base planes and labels of all pairs; region i belongs to pair img[i]
__global__ void k_pairwise_batch(DevPlanes P, KParams kp, const PairDesc *pairs, const int *img,
                                 const int4 *regions, const int64_t *offsets, const float4 *lab_all,
                                 const float *alpha, const float *costs_alpha, int32_t *tcaps, int32_t *ncaps,
                                 int64_t *cterm) {
    __shared__ long long red[33];
    const int i = blockIdx.x;
    const PairDesc pd = pairs[img[i]];
    pair_planes(P, kp, pd);
    const float4 *lab = lab_all + pd.off;
    const int4 R = regions[i];
    const float4 al = make_float4(alpha[3 * i], alpha[3 * i + 1], alpha[3 * i + 2], 0.f);
    const int n = R.z * R.w;
    const int64_t off = offsets[i];
    long long cst = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        NodeCaps o;
        build_node(P, kp, lab, al, costs_alpha[off + j], R.x, R.y, R.z, R.w, j % R.z, j / R.z, o);
        tcaps[2 * (off + j)] = o.cap_s;
        tcaps[2 * (off + j) + 1] = o.cap_t;
        for (int d = 0; d < 4; ++d) ncaps[4 * (off + j) + d] = o.k[d];
        cst += o.cst;
    }
    cst = block_sum_ll(cst, red);
    if (threadIdx.x == 0) cterm[i] = cst;
}

template <int NT>
__global__ void __launch_bounds__(NT, 1) k_mincut_batch(KParams kp, const int4 *regions, const int64_t *offsets,
                                                       const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                                                       int64_t *flow, int32_t *status, Counters *ctr) {
    extern __shared__ __align__(16) int smi[];
    __shared__ long long red[33];
    const int i = blockIdx.x;
    const int4 R = regions[i];
    const int n = R.z * R.w, w = R.z, h = R.w;
    const int64_t off = offsets[i];
    CutSmem cs = cut_layout(smi, n);
    RowCol rc(threadIdx.x, blockDim.x, w);
    for (int j = threadIdx.x; j < n; j += blockDim.x, rc.next()) {
        const int iy = rc.y, ix = rc.x;
        cs.v[j] = tcaps[2 * (off + j)] - tcaps[2 * (off + j) + 1];
        for (int k = 0; k < 8; ++k) {
            int c = 0;
            const int jx = ix + dir_dx(k), jy = iy + dir_dy(k);
            if (k < 4 && jx >= 0 && jx < w && jy >= 0 && jy < h) c = max(0, (int)ncaps[4 * (off + j) + k]);
            cs.res[k * n + j] = c;
        }
    }
    __syncthreads();
    clamp_terminals(n, w, h, cs.res, cs.v);
    __syncthreads();
    // flow into the sink = initial sink capacity - residual sink capacity at the end
    long long capt = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) capt += max(0, -cs.v[j]);
    capt = block_sum_ll(capt, red);
    CutCount cc{0, 0, 0};
    const int st = cta_maxflow(n, w, h, cs.res, cs.v, cs.hh, cs.bits, kp.max_rounds, kp.gr_interval, cc);
    long long rt = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        take[off + j] = (st == LEM_OK && cs.hh[j] != kInf) ? 1 : 0;
        rt += max(0, -cs.v[j]);
    }
    rt = block_sum_ll(rt, red);
    if (threadIdx.x == 0) {
        flow[i] = capt - rt;
        status[i] = st;
        atomicAdd(&ctr->rounds, (unsigned long long)cc.rounds);
        atomicAdd(&ctr->relabels, (unsigned long long)cc.relabels);
        atomicAdd(&ctr->bfs_levels, (unsigned long long)cc.levels);
    }
}

// One expansion move of region [x0, x0+w) x [y0, y0+h) with candidate al whose
// data term phi_p(al) is in `phi` (image plane, row pitch W): graph, terminal
// reduction, CTA min-cut, commit of the minimal sink side.  All threads call
// it; it ends with a barrier.
template <bool kOutline = false>
__device__ void expand_move(const DevPlanes &P, const KParams &kp, float4 *lab, const float *phi, float4 al, int x0,
                            int y0, int w, int h, const CutSmem &cs, CutCount &cc, long long &acc, long long &hits) {
    const int n = w * h, W = P.W;
    RowCol rb(threadIdx.x, blockDim.x, w);
    for (int j = threadIdx.x; j < n; j += blockDim.x, rb.next()) {
        const int iy = rb.y, ix = rb.x;
        NodeCaps o;
        build_node(P, kp, lab, al, phi[(size_t)(y0 + iy) * W + x0 + ix], x0, y0, w, h, ix, iy, o);
        cs.v[j] = o.cap_s - o.cap_t;
        for (int d = 0; d < 4; ++d) cs.res[d * n + j] = o.k[d];
        for (int d = 4; d < 8; ++d) cs.res[d * n + j] = 0;
    }
    __syncthreads();
    clamp_terminals(n, w, h, cs.res, cs.v);
    __syncthreads();
    const int st = cta_maxflow<kOutline>(n, w, h, cs.res, cs.v, cs.hh, cs.bits, kp.max_rounds, kp.gr_interval, cc);
    if (st == LEM_OK) {
        RowCol rm(threadIdx.x, blockDim.x, w);
        for (int j = threadIdx.x; j < n; j += blockDim.x, rm.next()) {
            if (cs.hh[j] == kInf) continue;
            const size_t p = (size_t)(y0 + rm.y) * W + x0 + rm.x;
            lab[p] = make_float4(al.x, al.y, al.z, phi[p]);
            ++acc;
        }
    } else if (threadIdx.x == 0) {
        ++hits;
    }
    __syncthreads();
}

// kind of proposal t of a visit (the order of Algorithm 2 with the learned
// proposer's map candidates): 0 propagation, 1 RANSAC, 2 map, 3 perturbation
__device__ __forceinline__ int proposal_kind(const Level &lv, int kc, int t) {
    return t < lv.k_prop ? 0 : (t < lv.k_prop + lv.k_rans ? 1 : (t < lv.k_prop + lv.k_rans + kc ? 2 : 3));
}

// block sums of the per-kind switched-pixel counts into the counters (all threads)
__device__ void add_accepted(const long long (&acck)[4], long long *red, Counters *ctr) {
    long long tot = 0;
    for (int k = 0; k < 4; ++k) {
        const long long s = block_sum_ll(acck[k], red);
        tot += s;
        if (threadIdx.x == 0 && s) atomicAdd(&ctr->accepted_kind[k], (unsigned long long)s);
    }
    if (threadIdx.x == 0) atomicAdd(&ctr->accepted, (unsigned long long)tot);
}

__device__ __forceinline__ bool same_label(float4 a, float4 b) {
    return __float_as_uint(a.x) == __float_as_uint(b.x) && __float_as_uint(a.y) == __float_as_uint(b.y) &&
           __float_as_uint(a.z) == __float_as_uint(b.z);
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Dataflow launches of a level.  The region of cell (ci, cj) covers cells
// ci - 1 .. ci + 1 (and rows likewise); its moves read the labels of the region
// and of the one-pixel ring around it and write the region's labels.  Two
// regions more than three cells apart in either direction therefore neither
// read nor write each other's pixels and their moves commute; regions closer
// than that must move in group order.  A region waits for the done flags of
// the cells of earlier groups within three cells (group index
// (cj & 3) * 4 + (ci & 3), the order of the 16 group launches) and sets its
// own flag after its last move.
// ---------------------------------------------------------------------------
constexpr int kDepWaitLimit = 1 << 24;  // polls, about 100 ns apart, before a wait gives up

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// all threads of the CTA; returns after the flags of the earlier-group cells
// within three cells of (ci, cj) are set (or their waits gave up, counted in
// ctr->dep_give_ups)
__device__ void wait_for_earlier_neighbours(const unsigned *done, int base, int ci, int cj, int nx, int ny,
                                            Counters *ctr) {
    const int t = threadIdx.x;
    if (t < 49) {
        const int x = ci + t % 7 - 3, y = cj + t / 7 - 3;
        const int g = ((cj & 3) << 2) | (ci & 3);
        if (x >= 0 && x < nx && y >= 0 && y < ny && ((((y & 3) << 2) | (x & 3)) < g)) {
            const unsigned *f = done + base + y * nx + x;
            int polls = 0;
            while (ld_acquire_gpu(f) == 0u) {
                if (++polls > kDepWaitLimit) {
                    atomicAdd(&ctr->dep_give_ups, 1ull);
                    break;
                }
                __nanosleep(100);
            }
        }
    }
    __syncthreads();
}

// all threads of the CTA, after the region's last move: publishes its label
// and cost writes and sets its done flag
__device__ void mark_region_done(unsigned *done, int idx) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(done + idx), "r"(1u) : "memory");
    }
}

// All expansions of one group at one level: one CTA per region, Algorithm 2.
//   P      : base planes of all pairs (H/W unused); pair b's planes start at
//            pixel pairs[b].off
//   items  : one (pair, cell i, cell j) per CTA (per CTA pair with phiB_all), or
//            with queue (two ints: next item, finished CTAs; zero before the
//            launch, zero again after it) taken from that work queue by a grid of
//            at most the co-resident CTAs until all n_items are done
//   iter   : outer iteration, or -1 to read it from *iter_dev (graph replay)
//   done   : NULL, or (with queue) the cells' done flags of a dataflow launch:
//            items are then all 16 groups of the level in group order and
//            item.w is the flag index of the pair's cell (0, 0)
//   SPEC   : a launch in clusters of two CTAs per region (phiB_all), for
//            levels whose visit is two propagation candidates (K_prop = 2, no
//            other proposals).  The second candidate is alpha_2 = f_r2 after
//            the first move, and the first move can only change f_r2 to
//            alpha_1; so CTA 1 computes phi(f_r2 before the move) into phiB
//            while CTA 0 computes phi(alpha_1), and after the first move CTA 0
//            redraws alpha_2 and takes its data term from phiB (unchanged f_r2)
//            or phiA (f_r2 = alpha_1).  With batched visits (K >= 2) both
//            candidates come from the visit-start labels and alpha_2 is the
//            first draw.  The moves and their results are those of the
//            one-CTA visit, bit for bit.
template <int NT, bool SPEC>
__global__ void __launch_bounds__(NT, NT <= 128 ? 4 : (NT <= 256 ? 3 : 1))
    k_expand_group(DevPlanes P0, KParams kp0, Level lv, int level, int iter, const int *iter_dev,
                   const PairDesc *pairs, const int4 *items, float4 *lab_all, float *phiA_all,
                   const float4 *prop_all, Counters *ctr, float *phiB_all, int n_items, int *queue,
                   unsigned *done) {
    extern __shared__ __align__(16) float smf[];
    __shared__ float4 s_alpha[kMaxVisit];
    __shared__ long long red[33];
    __shared__ int s_src;
    __shared__ int s_item;
    const int rank = SPEC ? (int)(blockIdx.x & 1u) : 0;
    if (iter < 0) iter = *iter_dev;
    long long acck[4] = {0, 0, 0, 0}, hits = 0;
    unsigned long long evals = 0;
    CutCount cc{0, 0, 0};
    // one item per CTA, or (queue) items taken from a work queue until none is left
    for (int pass = 0;; ++pass) {
    int idx;
    if (queue) {
        if (threadIdx.x == 0) s_item = atomicAdd(queue, 1);
        __syncthreads();
        idx = s_item;
        __syncthreads();
        if (idx >= n_items) break;
    } else {
        if (pass > 0) break;
        idx = SPEC ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    }
    const int4 item = items[idx];
    const PairDesc pd = pairs[item.x];
    DevPlanes P = P0;
    KParams kp = kp0;
    P.H = pd.H;
    P.W = pd.W;
    P.L = px_offset(P.L, pd.off, P.fmt);
    P.R = px_offset(P.R, pd.off, P.fmt);
    P.gst += 3 * pd.off;
    P.wfw += pd.off;
    kp.seed = pd.seed;
    kp.disp_min = pd.disp_min;
    kp.disp_max = pd.disp_max;
    float4 *lab = lab_all + pd.off;
    float *phiA = phiA_all + pd.off;
    const float4 *prop = prop_all ? prop_all + pd.off : nullptr;
    const int H = P.H, W = P.W, s = lv.s;
    const int ci = item.y, cj = item.z;
    const int x0 = max(0, (ci - 1) * s), x1 = min(W, (ci + 2) * s);
    const int y0 = max(0, (cj - 1) * s), y1 = min(H, (cj + 2) * s);
    const int w = x1 - x0, h = y1 - y0, n = w * h;
    const int cx0 = ci * s, cy0 = cj * s, cw = min(W, cx0 + s) - cx0, chh = min(H, cy0 + s) - cy0;
    const int nx = (W + s - 1) / s, ny = (H + s - 1) / s;
    if (!SPEC && done) wait_for_earlier_neighbours(done, item.w, ci, cj, nx, ny, ctr);
    CutSmem cs = cut_layout(smf, n);
    evals += (unsigned long long)n * (unsigned long long)(lv.k_prop + lv.k_rans + (prop ? lv.k_cnn : 0) + lv.k_rand);
    if constexpr (SPEC) {
        float *phiB = phiB_all + pd.off;
        const unsigned long long st1 = proposal_stream(kp.seed, iter, level, ci, cj, 0);
        const unsigned long long st2 = proposal_stream(kp.seed, iter, level, ci, cj, 1);
        if (threadIdx.x == 0) {
            s_alpha[0] = propose(lab, W, st1, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
            s_alpha[1] = propose(lab, W, st2, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
        }
        __syncthreads();
        const float4 a1 = s_alpha[0], a2s = s_alpha[1];
        if (rank == 1) {
            region_unary(P, kp, x0, y0, w, h, a2s.x, a2s.y, a2s.z, smf, phiB + (size_t)y0 * W + x0, W);
            cluster_sync_all();
            return;
        }
        region_unary(P, kp, x0, y0, w, h, a1.x, a1.y, a1.z, smf, phiA + (size_t)y0 * W + x0, W);
        cluster_sync_all();
        expand_move<(NT <= 256)>(P, kp, lab, phiA, a1, x0, y0, w, h, cs, cc, acck[0], hits);
        if (threadIdx.x == 0) {
            const float4 a2 = propose(lab, W, st2, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
            s_alpha[1] = a2;
            s_src = same_label(a2, a2s) ? 1 : (same_label(a2, a1) ? 0 : 2);
            if (kp.visit > 1) {
                // batched visits draw both candidates from the labels at the visit start
                s_alpha[1] = a2s;
                s_src = 1;
            }
        }
        __syncthreads();
        const float4 a2 = s_alpha[1];
        const int src = s_src;
        if (src == 2)  // (not reachable: the first move sets f_r2 to alpha_1 or keeps it)
            region_unary(P, kp, x0, y0, w, h, a2.x, a2.y, a2.z, smf, phiA + (size_t)y0 * W + x0, W);
        expand_move<(NT <= 256)>(P, kp, lab, src == 1 ? phiB : phiA, a2, x0, y0, w, h, cs, cc, acck[0], hits);
    } else {
        // outer perturbation sizes of this iteration, copied into Algorithm 2
        double rd = 0.5 * (kp.disp_max - kp.disp_min) * ldexp(1.0, -iter);
        double rn = ldexp(1.0, -iter);
        // proposal indices: [0, k_prop) propagation, then k_rans RANSAC planes, then
        // kc map candidates of the learned proposer, then k_rand perturbations
        const int kc = prop ? lv.k_cnn : 0, kr = lv.k_rans;
        const int nprop = lv.k_prop + kr + kc + lv.k_rand;
        const int K = kp.visit;
        for (int t0 = 0; t0 < nprop; t0 += K) {
            const int t1 = min(nprop, t0 + K);
            // the candidates of one visit, all drawn from the labels at its start
            // (K = 1: Algorithm 2 as printed): propagation, RANSAC (whole CTA), map
            // candidates, perturbation
            for (int t = t0; t < t1; ++t) {
                const unsigned long long stream = proposal_stream(kp.seed, iter, level, ci, cj, t);
                if (t >= lv.k_prop && t < lv.k_prop + kr) {
                    RansacSmem *rs = reinterpret_cast<RansacSmem *>(smf);
                    ransac_cta(lab, W, stream, cx0, cy0, cw, chh, rs, rs->dq, &s_alpha[t - t0]);
                    continue;
                }
                if (threadIdx.x != 0) continue;
                if (t >= lv.k_prop + kr && t < lv.k_prop + kr + kc) {
                    s_alpha[t - t0] = propose(prop, W, stream, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
                    continue;
                }
                const bool perturb = t >= lv.k_prop + kr + kc;
                s_alpha[t - t0] = propose(lab, W, stream, cx0, cy0, cw, chh, perturb, perturb ? rd : 0.0,
                                          perturb ? rn : 0.0, kp.disp_min, kp.disp_max);
                if (perturb) {
                    rd *= 0.5;
                    rn *= 0.5;
                }
            }
            __syncthreads();
            for (int t = t0; t < t1; ++t) {
                const float4 al = s_alpha[t - t0];
                region_unary(P, kp, x0, y0, w, h, al.x, al.y, al.z, smf, phiA + (size_t)y0 * W + x0, W);
                // (region_unary ends with a barrier; its shared memory is reused below)
                expand_move<(NT <= 256)>(P, kp, lab, phiA, al, x0, y0, w, h, cs, cc, acck[proposal_kind(lv, kc, t)],
                                         hits);
            }
        }
        if (done) mark_region_done(done, item.w + cj * nx + ci);
    }
    }
    add_accepted(acck, red, ctr);
    if (threadIdx.x == 0) {
        atomicAdd(&ctr->limit_hits, (unsigned long long)hits);
        atomicAdd(&ctr->evals, evals);
        atomicAdd(&ctr->rounds, (unsigned long long)cc.rounds);
        atomicAdd(&ctr->relabels, (unsigned long long)cc.relabels);
        atomicAdd(&ctr->bfs_levels, (unsigned long long)cc.levels);
        // the last CTA to finish resets the queue for the next launch (every CTA has
        // taken its last item before it counts itself done)
        if (queue && atomicAdd(queue + 1, 1) == (int)gridDim.x - 1) {
            queue[0] = 0;
            queue[1] = 0;
            __threadfence();
        }
    }
}

// ---------------------------------------------------------------------------
// Batched visits (K >= 2 candidates per visit, guided-filter data term, no
// RANSAC proposal): the candidates of a visit are all drawn from the labels at
// its start, so their data terms are independent of the visit's moves.  One
// visit of a (level, group) is then two launches:
//   k_visit_unary : one warp per (region, candidate): draws the candidate and
//                   computes its data term (warp_unary_gf) into plane t of phiK;
//   k_visit_cut   : one CTA per region: the K moves in candidate order, each
//                   against the labels the previous one left (graph, terminal
//                   reduction, push-relabel, commit).
// The moves, and so the labels, are those of the one-kernel visit; only the
// data term's summation differs (exact fixed-point sums here).
// ---------------------------------------------------------------------------
// the candidate of proposal t of a visit (lane 0 of the calling warp draws it;
// every lane gets it): propagation, map candidates, then perturbations whose
// size halves per perturbation of the region's Algorithm 2 call
__device__ __forceinline__ float4 visit_candidate(const KParams &kp, const Level &lv, int level, int iter, int ci,
                                                  int cj, int t, const float4 *lab, const float4 *prop, int W, int cx0,
                                                  int cy0, int cw, int chh) {
    float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
    if ((threadIdx.x & 31) == 0) {
        const unsigned long long stream = proposal_stream(kp.seed, iter, level, ci, cj, t);
        const int kc = prop ? lv.k_cnn : 0;
        if (t < lv.k_prop) {
            al = propose(lab, W, stream, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
        } else if (t < lv.k_prop + kc) {
            al = propose(prop, W, stream, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
        } else {
            const int np = t - lv.k_prop - kc;  // perturbations before this one
            const double rd = __dmul_rn(__dmul_rn(0.5 * (kp.disp_max - kp.disp_min), ldexp(1.0, -iter)),
                                        ldexp(1.0, -np));
            const double rn = __dmul_rn(ldexp(1.0, -iter), ldexp(1.0, -np));
            al = propose(lab, W, stream, cx0, cy0, cw, chh, true, rd, rn, kp.disp_min, kp.disp_max);
        }
    }
    al.x = __shfl_sync(kFull, al.x, 0);
    al.y = __shfl_sync(kFull, al.y, 0);
    al.z = __shfl_sync(kFull, al.z, 0);
    al.w = 0.f;
    return al;
}

// region of an item and its centre cell
struct ItemGeom {
    int x0, y0, w, h, cx0, cy0, cw, chh;
};
__device__ __forceinline__ ItemGeom item_geom(int ci, int cj, int s, int H, int W) {
    ItemGeom g;
    g.x0 = max(0, (ci - 1) * s);
    g.y0 = max(0, (cj - 1) * s);
    g.w = min(W, (ci + 2) * s) - g.x0;
    g.h = min(H, (cj + 2) * s) - g.y0;
    g.cx0 = ci * s;
    g.cy0 = cj * s;
    g.cw = min(W, g.cx0 + s) - g.cx0;
    g.chh = min(H, g.cy0 + s) - g.cy0;
    return g;
}


//   units: n_items * nK, unit u = (item u / nK, proposal t0 + u % nK)
//   phiK : nK planes of plane_stride floats (every pair's pixels); alphaK[u]
template <int NC>
__global__ void __launch_bounds__(128) k_visit_unary(DevPlanes P, KParams kp, Level lv, int level, int iter,
                                                     const int *iter_dev, const PairDesc *pairs, const int4 *items,
                                                     int n_items, int t0, int nK, const float4 *lab_all,
                                                     float *phiK, long long plane_stride, const float4 *prop_all,
                                                     float4 *alphaK, int mwp, int kwp) {
    extern __shared__ __align__(16) float smw[];
    const int warp = threadIdx.x >> 5;
    const int unit = blockIdx.x * (blockDim.x >> 5) + warp;
    if (unit >= n_items * nK) return;  // the whole warp leaves together
    const int it = unit / nK, t = unit - it * nK;
    const int4 item = items[it];
    const PairDesc pd = pairs[item.x];
    pair_planes(P, kp, pd);
    if (iter < 0) iter = *iter_dev;
    const ItemGeom g = item_geom(item.y, item.z, lv.s, P.H, P.W);
    const float4 *lab = lab_all + pd.off;
    const float4 *prop = prop_all ? prop_all + pd.off : nullptr;
    const float4 al = visit_candidate(kp, lv, level, iter, item.y, item.z, t0 + t, lab, prop, P.W, g.cx0, g.cy0, g.cw,
                                      g.chh);
    if ((threadIdx.x & 31) == 0) alphaK[unit] = al;
    float *ring = smw + (size_t)warp * warp_ring_floats(kp.r, mwp, kwp);
    float *out = phiK + (size_t)t * plane_stride + pd.off + (size_t)g.y0 * P.W + g.x0;
    warp_unary_gf<NC>(P, kp, g.x0, g.y0, g.w, g.h, al.x, al.y, al.z, ring, mwp, kwp, out, P.W);
}

// lem_unary_batch on handles with batched visits: the warp data term of the
// expansion path, one warp per (region, label)
template <int NC>
__global__ void __launch_bounds__(128) k_unary_batch_warp(DevPlanes P, KParams kp, const PairDesc *pairs,
                                                          const int *img, const int4 *regions,
                                                          const int64_t *offsets, int n_regions, int K,
                                                          const float *labels, float *costs, int mwp, int kwp) {
    extern __shared__ __align__(16) float smw[];
    const int warp = threadIdx.x >> 5;
    const int unit = blockIdx.x * (blockDim.x >> 5) + warp;
    if (unit >= n_regions * K) return;
    const int i = unit / K, k = unit - i * K;
    pair_planes(P, kp, pairs[img[i]]);
    const int4 R = regions[i];
    const float *l = labels + (size_t)unit * 3;
    float *out = costs + offsets[i] + (int64_t)k * R.z * R.w;
    warp_unary_gf<NC>(P, kp, R.x, R.y, R.z, R.w, l[0], l[1], l[2],
                      smw + (size_t)warp * warp_ring_floats(kp.r, mwp, kwp), mwp, kwp, out, R.z);
}

template <int NT>
__global__ void __launch_bounds__(NT, NT >= 512 ? 1 : 512 / NT)
    k_visit_cut(DevPlanes P, KParams kp, Level lv, const PairDesc *pairs, const int4 *items, int t0, int nK, int kc,
                float4 *lab_all, const float *phiK, long long plane_stride, const float4 *alphaK, Counters *ctr) {
    extern __shared__ __align__(16) float smf[];
    __shared__ long long red[33];
    const int4 item = items[blockIdx.x];
    const PairDesc pd = pairs[item.x];
    pair_planes(P, kp, pd);
    const ItemGeom g = item_geom(item.y, item.z, lv.s, P.H, P.W);
    const int n = g.w * g.h;
    float4 *lab = lab_all + pd.off;
    CutSmem cs = cut_layout(smf, n);
    long long acck[4] = {0, 0, 0, 0}, hits = 0;
    CutCount cc{0, 0, 0};
    for (int t = 0; t < nK; ++t) {
        const float4 al = alphaK[(size_t)blockIdx.x * nK + t];
        expand_move(P, kp, lab, phiK + (size_t)t * plane_stride + pd.off, al, g.x0, g.y0, g.w, g.h, cs, cc,
                    acck[proposal_kind(lv, kc, t0 + t)], hits);
    }
    add_accepted(acck, red, ctr);
    if (threadIdx.x == 0) {
        atomicAdd(&ctr->limit_hits, (unsigned long long)hits);
        atomicAdd(&ctr->evals, (unsigned long long)n * (unsigned long long)nK);
        atomicAdd(&ctr->rounds, (unsigned long long)cc.rounds);
        atomicAdd(&ctr->relabels, (unsigned long long)cc.relabels);
        atomicAdd(&ctr->bfs_levels, (unsigned long long)cc.levels);
    }
}

// ---------------------------------------------------------------------------
// learned-proposer glue: quarter-resolution features / targets of a label map
// and full-resolution plane proposals from the network's output
// ---------------------------------------------------------------------------
__global__ void k_cnn_features(DevPlanes P, const float4 *lab, int H4, int W4, float inv_dmax, float *x) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= H4 * W4) return;
    const int U = q % W4, V = q / W4;
    float s[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int cnt = 0;
    for (int dy = 0; dy < 4; ++dy)
        for (int dx = 0; dx < 4; ++dx) {
            const int u = 4 * U + dx, v = 4 * V + dy;
            if (u >= P.W || v >= P.H) continue;
            const size_t p = (size_t)v * P.W + u;
            const float4 l = load_px(P.L, p, P.fmt), r = load_px(P.R, p, P.fmt), f = lab[p];
            s[0] += l.x;
            s[1] += l.y;
            s[2] += l.z;
            s[3] += r.x;
            s[4] += r.y;
            s[5] += r.z;
            s[6] += fmaf(f.x, (float)u, fmaf(f.y, (float)v, f.z));
            ++cnt;
        }
    const float inv = 1.f / (float)cnt;
    for (int c = 0; c < 6; ++c) x[(size_t)q * 7 + c] = s[c] * inv * (1.f / 255.f);
    x[(size_t)q * 7 + 6] = s[6] * inv * inv_dmax;
}

__global__ void k_cnn_targets(const float4 *lab, int H, int W, int H4, int W4, float inv_dmax, float *t) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= H4 * W4) return;
    const int U = q % W4, V = q / W4;
    float d = 0.f, a = 0.f, b = 0.f;
    int cnt = 0;
    for (int dy = 0; dy < 4; ++dy)
        for (int dx = 0; dx < 4; ++dx) {
            const int u = 4 * U + dx, v = 4 * V + dy;
            if (u >= W || v >= H) continue;
            const float4 f = lab[(size_t)v * W + u];
            d += fmaf(f.x, (float)u, fmaf(f.y, (float)v, f.z));
            a += f.x;
            b += f.y;
            ++cnt;
        }
    // slopes beyond 1 (more than a pixel of disparity per pixel) are clamped: such
    // labels are left-overs of the random initialisation, not surfaces to learn
    const float inv = 1.f / (float)cnt;
    t[(size_t)q * 3] = d * inv * inv_dmax;
    t[(size_t)q * 3 + 1] = fminf(fmaxf(a * inv, -1.f), 1.f);
    t[(size_t)q * 3 + 2] = fminf(fmaxf(b * inv, -1.f), 1.f);
}

// bilinear interpolation of (d/dmax, a, b) at the pixel centre (quarter-
// resolution cell U covers pixels 4U .. 4U+3, centre 4U + 1.5), then
// c = d - a u - b v
__global__ void k_cnn_upsample(const float *y, int H4, int W4, int H, int W, float dmax, float4 *prop) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    const int u = p % W, v = p / W;
    const float fu = fminf(fmaxf(((float)u - 1.5f) * 0.25f, 0.f), (float)(W4 - 1));
    const float fv = fminf(fmaxf(((float)v - 1.5f) * 0.25f, 0.f), (float)(H4 - 1));
    const int u0 = (int)fu, v0 = (int)fv;
    const int u1 = min(u0 + 1, W4 - 1), v1 = min(v0 + 1, H4 - 1);
    const float tu = fu - (float)u0, tv = fv - (float)v0;
    float r[3];
    for (int c = 0; c < 3; ++c) {
        const float a00 = y[((size_t)v0 * W4 + u0) * 3 + c], a01 = y[((size_t)v0 * W4 + u1) * 3 + c];
        const float a10 = y[((size_t)v1 * W4 + u0) * 3 + c], a11 = y[((size_t)v1 * W4 + u1) * 3 + c];
        const float top = fmaf(tu, a01 - a00, a00), bot = fmaf(tu, a11 - a10, a10);
        r[c] = fmaf(tv, bot - top, top);
    }
    const float d = r[0] * dmax, a = r[1], b = r[2];
    prop[p] = make_float4(a, b, d - a * (float)u - b * (float)v, 0.f);
}

__global__ void k_props_in(int n, const float *abc, float4 *prop) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n) prop[p] = make_float4(abc[3 * (size_t)p], abc[3 * (size_t)p + 1], abc[3 * (size_t)p + 2], 0.f);
}

// ---------------------------------------------------------------------------
// post-processing: left-right consistency, occlusion filling, weighted median
// (Sec. 3.4, after Bleyer et al. 2011).  Disparities are (a u + b v) + c in FP32
// with one rounding per operation.  The right view's labels come from a handle
// on the mirrored pair: right pixel u is mirrored column W - 1 - u.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float plane_disp(const float4 &f, int u, int v) {
    return __fadd_rn(__fadd_rn(__fmul_rn(f.x, (float)u), __fmul_rn(f.y, (float)v)), f.z);
}

__global__ void k_lr_check(const float4 *labL, const float4 *labRm, int H, int W, float thr, uint8_t *valid) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    const int u = p % W, v = p / W;
    const float dL = plane_disp(labL[p], u, v);
    const float qf = rintf(__fsub_rn((float)u, dL));
    bool ok = false;
    if (qf >= 0.f && qf <= (float)(W - 1)) {
        const int q = (int)qf, um = W - 1 - q;
        const float dR = plane_disp(labRm[(size_t)v * W + um], um, v);
        ok = fabsf(__fsub_rn(dL, dR)) <= thr;
    }
    valid[p] = ok ? 1 : 0;
}

// filled disparity of every pixel: its own where consistent, else the lower of the
// planes of the nearest consistent pixels to its left and right on the row
__global__ void k_fill(const float4 *labL, const uint8_t *valid, int H, int W, float *disp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    const int u = p % W, v = p / W;
    const size_t row = (size_t)v * W;
    if (valid[p]) {
        disp[p] = plane_disp(labL[p], u, v);
        return;
    }
    float best = 0.f;
    bool have = false;
    int k = u - 1;
    while (k >= 0 && !valid[row + k]) --k;
    if (k >= 0) {
        best = plane_disp(labL[row + k], u, v);
        have = true;
    }
    k = u + 1;
    while (k < W && !valid[row + k]) ++k;
    if (k < W) {
        const float d = plane_disp(labL[row + k], u, v);
        best = have ? fminf(best, d) : d;
        have = true;
    }
    disp[p] = have ? best : plane_disp(labL[p], u, v);
}

// order-preserving map of a float to an unsigned key
__device__ __forceinline__ uint32_t fkey(float x) {
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float fkey_inv(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// one warp per inconsistent pixel: the smallest window value whose cumulative
// colour weight reaches half the total, found by bisection on the value keys
__global__ void k_wmedian(DevPlanes P, const uint8_t *valid, const float *disp, int radius, float inv_gamma,
                          float *out) {
    const int H = P.H, W = P.W;
    const int lane = threadIdx.x & 31;
    const int p = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (p >= H * W) return;
    if (valid[p]) {
        if (lane == 0) out[p] = disp[p];
        return;
    }
    const int u = p % W, v = p / W;
    const int x0 = max(0, u - radius), x1 = min(W - 1, u + radius);
    const int y0 = max(0, v - radius), y1 = min(H - 1, v + radius);
    const int ww = x1 - x0 + 1, cnt = ww * (y1 - y0 + 1);
    const float4 c = load_px(P.L, p, P.fmt);
    // total weight and the value range
    float tot = 0.f;
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    for (int j = lane; j < cnt; j += 32) {
        const int yy = y0 + j / ww, xx = x0 + j % ww;
        const size_t q = (size_t)yy * W + xx;
        const float4 cq = load_px(P.L, q, P.fmt);
        const float l1 = fabsf(cq.x - c.x) + fabsf(cq.y - c.y) + fabsf(cq.z - c.z);
        tot += expf(-l1 * inv_gamma);
        const uint32_t k = fkey(disp[q]);
        kmin = min(kmin, k);
        kmax = max(kmax, k);
    }
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    const float half = 0.5f * tot;
    // smallest key k in [kmin, kmax] with weight(<= k) >= half
    uint32_t lo = kmin, hi = kmax;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        float s = 0.f;
        for (int j = lane; j < cnt; j += 32) {
            const int yy = y0 + j / ww, xx = x0 + j % ww;
            const size_t q = (size_t)yy * W + xx;
            if (fkey(disp[q]) <= mid) {
                const float4 cq = load_px(P.L, q, P.fmt);
                s += expf(-(fabsf(cq.x - c.x) + fabsf(cq.y - c.y) + fabsf(cq.z - c.z)) * inv_gamma);
            }
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (s >= half)
            hi = mid;
        else
            lo = mid + 1;
    }
    if (lane == 0) out[p] = fkey_inv(lo);
}

__global__ void k_props_out(int n, const float4 *prop, float *abc) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const float4 f = prop[p];
    abc[3 * (size_t)p] = f.x;
    abc[3 * (size_t)p + 1] = f.y;
    abc[3 * (size_t)p + 2] = f.z;
}

// The candidates of one visit of each listed cell, drawn from the current labels
// as k_expand_group draws them (no moves in between): one CTA per cell.
//   cells: (ci, cj) per CTA; alpha: per cell, nprop labels (a, b, c)
__global__ void k_propose_batch(DevPlanes P, KParams kp, Level lv, int level, int iter, const int2 *cells,
                                const float4 *lab, const float4 *prop, float *alpha, long long *dq_g) {
    extern __shared__ __align__(16) float smf[];
    __shared__ float4 s_one;
    const int W = P.W, H = P.H, s = lv.s;
    const int ci = cells[blockIdx.x].x, cj = cells[blockIdx.x].y;
    const int cx0 = ci * s, cy0 = cj * s, cw = min(W, cx0 + s) - cx0, chh = min(H, cy0 + s) - cy0;
    double rd = 0.5 * (kp.disp_max - kp.disp_min) * ldexp(1.0, -iter);
    double rn = ldexp(1.0, -iter);
    const int kc = prop ? lv.k_cnn : 0, kr = lv.k_rans;
    const int nprop = lv.k_prop + kr + kc + lv.k_rand;
    for (int t = 0; t < nprop; ++t) {
        const unsigned long long stream = proposal_stream(kp.seed, iter, level, ci, cj, t);
        if (t >= lv.k_prop && t < lv.k_prop + kr) {
            RansacSmem *rs = reinterpret_cast<RansacSmem *>(smf);
            ransac_cta(lab, W, stream, cx0, cy0, cw, chh, rs, dq_g ? dq_g + (size_t)blockIdx.x * s * s : rs->dq,
                       &s_one);
        } else if (threadIdx.x == 0) {
            if (t >= lv.k_prop + kr && t < lv.k_prop + kr + kc) {
                s_one = propose(prop, W, stream, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
            } else {
                const bool perturb = t >= lv.k_prop + kr + kc;
                s_one = propose(lab, W, stream, cx0, cy0, cw, chh, perturb, perturb ? rd : 0.0, perturb ? rn : 0.0,
                                kp.disp_min, kp.disp_max);
                if (perturb) {
                    rd *= 0.5;
                    rn *= 0.5;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float *o = alpha + ((size_t)blockIdx.x * nprop + t) * 3;
            o[0] = s_one.x;
            o[1] = s_one.y;
            o[2] = s_one.z;
        }
        __syncthreads();
    }
}

// A9: quantised energy, per-block partial sums
__global__ void k_energy(DevPlanes P, KParams kp, const float4 *lab, long long *partials) {
    __shared__ long long red[33];
    const int H = P.H, W = P.W;
    long long e = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < H * W; p += gridDim.x * blockDim.x) {
        const int x = p % W, y = p / W;
        const float4 f = lab[p];
        e += q_cost(f.w, kp.S);
        const float4 wp = P.wfw[p];
        for (int d = 0; d < 4; ++d) {
            const int qx = x + dir_dx(d), qy = y + dir_dy(d);
            if (qx < 0 || qx >= W || qy >= H) continue;
            e += q_psi(comp(wp, d), kp.tau_dis, kp.S, f, lab[(size_t)qy * W + qx], x, y, qx, qy);
        }
    }
    e = block_sum_ll(e, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = e;
}

__global__ void k_sum_partials(const long long *partials, int n, long long *out) {
    __shared__ long long red[33];
    long long s = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
    s = block_sum_ll(s, red);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_labels_out(int H, int W, const float4 *lab, float *abc, float *disp, float *cost) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    const float4 f = lab[p];
    if (abc) {
        abc[3 * p] = f.x;
        abc[3 * p + 1] = f.y;
        abc[3 * p + 2] = f.z;
    }
    if (disp) disp[p] = fmaf(f.x, (float)(p % W), fmaf(f.y, (float)(p / W), f.z));
    if (cost) cost[p] = f.w;
}

__global__ void k_labels_in(int H, int W, const float *abc, const float *cost, float4 *lab) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    lab[p] = make_float4(abc[3 * p], abc[3 * p + 1], abc[3 * p + 2], cost ? cost[p] : 0.f);
}

__global__ void k_planes_out(int H, int W, DevPlanes P, float *left, float *right, float *guide, float *weights) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= H * W) return;
    if (left) reinterpret_cast<float4 *>(left)[p] = load_px(P.L, p, P.fmt);
    if (right) reinterpret_cast<float4 *>(right)[p] = load_px(P.R, p, P.fmt);
    if (weights) reinterpret_cast<float4 *>(weights)[p] = P.wfw[p];
    if (guide) {
        const float4 a = P.gst[3 * p], b = P.gst[3 * p + 1], c = P.gst[3 * p + 2];
        float *g = guide + 9 * (size_t)p;
        g[0] = a.x;
        g[1] = a.y;
        g[2] = a.z;
        g[3] = a.w;
        g[4] = b.x;
        g[5] = b.y;
        g[6] = b.z;
        g[7] = b.w;
        g[8] = c.x;
    }
}

// ---------------------------------------------------------------------------
// Regions above the shared-memory cut.  With cells proportional to the image
// width (Sec. 4, Middlebury V3: 1, 3 and 9 % of the width) a 3x3-cell region
// reaches 135x135 or 405x405 nodes at 1500 px.  Such a region is spread over
// G CTAs of one cooperative launch (all co-resident): its graph, heights and
// relabel bitplanes live in a global slot (L2-resident), the data term runs
// on 64x128 tiles spread over the CTAs, and the CTAs meet at region barriers.
// The cut is the same canonical minimal sink side as the CTA cut's.
// ---------------------------------------------------------------------------
constexpr int kGridTileW = 64, kGridTileH = 128;
constexpr int kGridInf = 0x3fffffff;
constexpr long long kRegionWaitNs = 1000000000ll;  // a region barrier gives up after 1 s
constexpr int kGridThreads = 512;
constexpr int kGridUnroll = 4;  // compaction: 4 x 4 nodes per thread per pass

struct RegionSync {
    // one word per barrier generation mod 3: arrivals in the high 32 bits, the
    // sum of the values the CTAs bring in the low 32
    unsigned long long slot[3];
    int err;  // set by a CTA whose barrier gave up (diagnostics)
    int pad;
    float4 alpha[kMaxVisit];  // candidates of the current visit
};

// ints of one region slot for regions up to w x h nodes: residuals (8n),
// then excess, heights and the active list (n4 = n rounded up to 4 each, so
// every array starts on 16 bytes), then the relabel bitplanes (11 h WPR
// words); rounded to 256 bytes
__host__ __device__ inline long long grid_slot_ints(int w, int h) {
    const long long n = (long long)w * h, n4 = (n + 3) & ~3ll, wpr = (w + 31) / 32;
    return (8 * n + 3 * n4 + 11 * h * wpr + 63) & ~63ll;
}

// the arrays of a region of n nodes in its slot
struct GridSlot {
    int *res, *v, *hh, *list;
    uint32_t *bits;
};
__device__ __forceinline__ GridSlot grid_slot(int *base, int n) {
    const size_t n4 = ((size_t)n + 3) & ~(size_t)3;
    GridSlot g;
    g.res = base;
    g.v = base + 8 * (size_t)n;
    g.hh = g.v + n4;
    g.list = g.hh + n4;
    g.bits = reinterpret_cast<uint32_t *>(g.list + n4);
    return g;
}

// node range [i0, i1) of CTA c of G: boundaries on multiples of 4 (the last range ends at n)
__device__ __forceinline__ int grid_range_start(int n, int c, int G) {
    return c >= G ? n : (int)(((long long)n * c / G) & ~3ll);
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// the CTA's place in its region and the barrier state
struct RegionCtx {
    RegionSync *rs;
    int G, c;
    unsigned gen;  // barriers passed (the same in every thread of every CTA of the region)
    int *s_flag;   // shared: this CTA gave up at a barrier
    int *s_val;    // shared: result of the last barrier
};

// Barrier of the G CTAs of one region that also sums `val` (thread 0's value
// of each CTA); every thread calls it and gets the sum, or -1 once this CTA's
// wait gave up (1 s without all arrivals; every later barrier of the CTA then
// returns -1 at once, and the other CTAs give up at their next barrier).
// Thread 0 arrives with a release reduction on the generation's word and
// polls it with acquire loads: writes before the barrier in any CTA of the
// region are visible after it in every CTA.
__device__ int region_step(RegionCtx &x, int val) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int out = -1;
        if (!*x.s_flag) {
            unsigned long long *w = &x.rs->slot[x.gen % 3];
            red_release_add_u64(w, (1ull << 32) + (unsigned)val);
            const unsigned long long need = (unsigned long long)x.G << 32;
            unsigned long long cur = ld_acquire_u64(w);
            long long t0 = 0;
            for (int k = 0; cur < need; ++k) {
                if ((k & 63) == 63) {
                    const long long t = global_ns();
                    if (t0 == 0) {
                        t0 = t;
                    } else if (t - t0 > kRegionWaitNs) {
                        atomicExch(&x.rs->err, 1);
                        *x.s_flag = 1;
                        break;
                    }
                }
                cur = ld_acquire_u64(w);
            }
            if (cur >= need) {
                out = (int)(cur & 0xffffffffull);
                // the word of the barrier two ahead: its last readers have all arrived here
                if (x.c == 0) x.rs->slot[(x.gen + 2) % 3] = 0ull;
            }
        }
        *x.s_val = out;
    }
    ++x.gen;
    __syncthreads();
    return *x.s_val;
}

__device__ __forceinline__ bool region_sync(RegionCtx &x) { return region_step(x, 0) >= 0; }
__device__ __forceinline__ int region_sum(RegionCtx &x, int val) { return region_step(x, val); }

// Exact distances to the sink, by the bit-parallel BFS of global_relabel with
// the bitplanes in global memory: CTA c builds and scans the row words
// [NW c / G, NW (c+1) / G) and every BFS level ends with a region barrier.
// Returns 1 when a node with excess reaches the sink, 0 when none does, -1
// when a barrier gave up.
__device__ int grid_relabel(int n, int w, int h, const int *res, const int *v, int *hh, uint32_t *bits, int i0,
                            int i1, RegionCtx &x, int *levels) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    const int WPR = (w + 31) >> 5, NW = h * WPR;
    const int wb0 = (int)((long long)NW * x.c / x.G), wb1 = (int)((long long)NW * (x.c + 1) / x.G);
    uint32_t *M = bits, *Fa = bits + 8 * (size_t)NW, *Fb = Fa + NW, *VIS = Fb + NW;
    for (int word = wb0 + warp; word < wb1; word += nwarp) {
        const int y = word / WPR, wi = word - y * WPR;
        const int xx = wi * 32 + lane;
        const bool in = xx < w;
        const int i = y * w + xx;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            bool pred = false;
            if (in) pred = res[(size_t)k * n + i] > 0;
            const uint32_t m = __ballot_sync(0xffffffffu, pred);
            if (lane == 0) M[(size_t)k * NW + word] = m;
        }
        bool seed = false;
        if (in) seed = v[i] < 0;
        const uint32_t m = __ballot_sync(0xffffffffu, seed);
        if (lane == 0) {
            Fa[word] = m;
            VIS[word] = m;
        }
        if (in) hh[i] = seed ? 1 : kGridInf;
    }
    if (!region_sync(x)) return -1;
    uint32_t *Fc = Fa, *Fn = Fb;
    int level = 1;
    for (;;) {
        int any = 0;
        for (int word = wb0 + tid; word < wb1; word += nt) {
            const int y = word / WPR, wi = word - y * WPR;
            const uint32_t vis = VIS[word];
            uint32_t cand = 0;
            if (~vis) {
                uint32_t sh[3][3];
#pragma unroll
                for (int r = 0; r < 3; ++r) {
                    const int yy = y + r - 1;
                    uint32_t cw = 0, lw = 0, rw = 0;
                    if (yy >= 0 && yy < h) {
                        const uint32_t *F = Fc + (size_t)yy * WPR;
                        cw = F[wi];
                        lw = wi > 0 ? F[wi - 1] : 0u;
                        rw = wi + 1 < WPR ? F[wi + 1] : 0u;
                    }
                    sh[r][0] = (cw << 1) | (lw >> 31);
                    sh[r][1] = cw;
                    sh[r][2] = (cw >> 1) | (rw << 31);
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) cand |= M[(size_t)k * NW + word] & sh[dir_dy(k) + 1][dir_dx(k) + 1];
                const int tail = w - wi * 32;
                cand &= ~vis & (tail >= 32 ? 0xffffffffu : ((1u << tail) - 1u));
            }
            Fn[word] = cand;
            if (cand) {
                VIS[word] = vis | cand;
                any = 1;
                uint32_t cc = cand;
                const int base = y * w + wi * 32;
                while (cc) {
                    const int b = __ffs(cc) - 1;
                    cc &= cc - 1;
                    hh[base + b] = level + 1;
                }
            }
        }
        any = __syncthreads_or(any);
        const int tot = region_sum(x, any);
        if (tot < 0) return -1;
        if (tot == 0) break;
        uint32_t *t = Fc;
        Fc = Fn;
        Fn = t;
        ++level;
    }
    *levels += level;
    int act = 0;
    for (int i = i0 + tid; i < i1; i += nt) act |= (v[i] > 0 && hh[i] != kGridInf);
    act = __syncthreads_or(act);
    const int tot = region_sum(x, act);
    return tot < 0 ? -1 : (tot > 0 ? 1 : 0);
}

// Terminal reduction of clamp_terminals for the nodes [i0, i1) of the CTA.
__device__ void grid_clamp_terminals(int n, int w, int h, const int *res, int *v, int i0, int i1) {
    for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const int e = v[i];
        if (e > 0) {
            int out = 1;
#pragma unroll
            for (int k = 0; k < 8; ++k) out += res[(size_t)k * n + i];
            v[i] = min(e, out);
        } else if (e < 0) {
            const int iy = i / w, ix = i - iy * w;
            int in = 1;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int jx = ix + dir_dx(k), jy = iy + dir_dy(k);
                if (jx < 0 || jx >= w || jy < 0 || jy >= h) continue;
                in += res[(size_t)(k ^ 4) * n + i + dir_off(k, w)];
            }
            v[i] = max(e, -in);
        }
    }
}

// Maximum preflow of the region, rounds as in cta_maxflow: each CTA compacts
// and pushes its own nodes [i0, i1) (pushes into other CTAs' nodes are device
// atomics), and a round ends with a region barrier that also sums the active
// counts.  LEM_OK: hh[i] != kGridInf exactly on the minimal sink side;
// LEM_ERR_MAXFLOW_LIMIT, or LEM_ERR_CUDA when a barrier gave up.
__device__ int grid_maxflow(int n, int w, int h, int *res, int *v, int *hh, int *list, uint32_t *bits, int i0,
                            int i1, int max_rounds, int gr_interval, RegionCtx &x, CutCount &cc, int *s_cnt) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    int act = grid_relabel(n, w, h, res, v, hh, bits, i0, i1, x, &cc.levels);
    ++cc.relabels;
    if (act < 0) return LEM_ERR_CUDA;
    int rounds = 0;
    while (act) {
        if (rounds >= max_rounds) {
            cc.rounds += rounds;
            return LEM_ERR_MAXFLOW_LIMIT;
        }
        if (tid == 0) *s_cnt = 0;
        __syncthreads();
        // 4 consecutive nodes per thread and kGridUnroll such groups per pass,
        // every load of a pass issued before the first append (the node range
        // starts on a multiple of 4, the arrays on 16 bytes)
        for (int base = i0; base < i1; base += 4 * kGridUnroll * nt) {
            int4 vv[kGridUnroll], h4[kGridUnroll];
#pragma unroll
            for (int u = 0; u < kGridUnroll; ++u) {
                const int j = base + 4 * (u * nt + tid);
                vv[u] = make_int4(0, 0, 0, 0);
                h4[u] = make_int4(kGridInf, kGridInf, kGridInf, kGridInf);
                if (j + 3 < i1) {
                    vv[u] = *reinterpret_cast<const int4 *>(v + j);
                    h4[u] = *reinterpret_cast<const int4 *>(hh + j);
                } else if (j < i1) {
                    vv[u].x = v[j];
                    h4[u].x = hh[j];
                    if (j + 1 < i1) {
                        vv[u].y = v[j + 1];
                        h4[u].y = hh[j + 1];
                    }
                    if (j + 2 < i1) {
                        vv[u].z = v[j + 2];
                        h4[u].z = hh[j + 2];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kGridUnroll; ++u) {
                const int j = base + 4 * (u * nt + tid);
                const bool a0 = vv[u].x > 0 && h4[u].x != kGridInf, a1 = vv[u].y > 0 && h4[u].y != kGridInf;
                const bool a2 = vv[u].z > 0 && h4[u].z != kGridInf, a3 = vv[u].w > 0 && h4[u].w != kGridInf;
                const int cnt4 = (int)a0 + (int)a1 + (int)a2 + (int)a3;
                int incl = cnt4;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int tot = __shfl_sync(0xffffffffu, incl, 31);
                if (tot == 0) continue;
                int pos = 0;
                if (lane == 31) pos = atomicAdd(s_cnt, tot);
                pos = __shfl_sync(0xffffffffu, pos, 31) + incl - cnt4;
                int *L = list + i0;
                if (a0) L[pos++] = j;
                if (a1) L[pos++] = j + 1;
                if (a2) L[pos++] = j + 2;
                if (a3) L[pos] = j + 3;
            }
        }
        __syncthreads();
        const int cnt = *s_cnt;
        for (int q = tid; q < cnt; q += nt) {
            const int i = list[i0 + q];
            const int e = v[i];
            const int hu = hh[i];
            int r[8], hn[8];
            // residuals and neighbour heights loaded together (neighbours by position)
            const int iy = i / w, ix = i - iy * w;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                r[k] = res[(size_t)k * n + i];
                const int jx = ix + dir_dx(k), jy = iy + dir_dy(k);
                hn[k] = (jx >= 0 && jx < w && jy >= 0 && jy < h) ? hh[i + dir_off(k, w)] : kGridInf;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (r[k] <= 0) hn[k] = kGridInf;
            int left = e, mh = kGridInf;
            int d[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                d[k] = 0;
                if (r[k] > 0 && hn[k] + 1 == hu && left > 0) {
                    d[k] = min(left, r[k]);
                    left -= d[k];
                }
                if (r[k] - d[k] > 0) mh = min(mh, hn[k]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (d[k] == 0) continue;
                const int j = i + dir_off(k, w);
                atomicSub(&res[(size_t)k * n + i], d[k]);
                atomicAdd(&res[(size_t)(k ^ 4) * n + j], d[k]);
                atomicAdd(&v[j], d[k]);
            }
            if (left != e) atomicSub(&v[i], e - left);
            if (left > 0) hh[i] = (mh >= n + 1) ? kGridInf : mh + 1;
        }
        ++rounds;
        const int tot = region_sum(x, cnt);
        if (tot < 0) return LEM_ERR_CUDA;
        if (tot == 0 || rounds % gr_interval == 0) {
            act = grid_relabel(n, w, h, res, v, hh, bits, i0, i1, x, &cc.levels);
            ++cc.relabels;
            if (act < 0) return LEM_ERR_CUDA;
        }
    }
    cc.rounds += rounds;
    return LEM_OK;
}

// All expansions of one group at one level for regions above the shared-memory
// cut: G CTAs per region (blockIdx.x = region * G + c), Algorithm 2 as in
// k_expand_group.  CTA 0 of a region draws the candidates of a visit; the data
// term runs on tiles; each CTA builds, clamps and commits its own node range.
//   slots: one global slot of slot_ints ints per region of the launch
//   sync : one zeroed RegionSync per region of the launch
template <int NT>
__global__ void __launch_bounds__(NT, 1)
    k_expand_grid(DevPlanes P, KParams kp, Level lv, int level, int iter, int G, const PairDesc *pairs,
                  const int4 *items, float4 *lab_all, float *phiA_all, const float4 *prop_all, int *slots,
                  long long slot_ints, RegionSync *sync, Counters *ctr) {
    extern __shared__ __align__(16) float smf[];
    __shared__ float4 s_alpha[kMaxVisit];
    __shared__ long long red[33];
    __shared__ int s_flag, s_val, s_cnt;
    const int ridx = blockIdx.x / G, c = blockIdx.x - ridx * G;
    const int4 item = items[ridx];
    const PairDesc pd = pairs[item.x];
    P.H = pd.H;
    P.W = pd.W;
    P.L = px_offset(P.L, pd.off, P.fmt);
    P.R = px_offset(P.R, pd.off, P.fmt);
    P.gst += 3 * pd.off;
    P.wfw += pd.off;
    kp.seed = pd.seed;
    kp.disp_min = pd.disp_min;
    kp.disp_max = pd.disp_max;
    float4 *lab = lab_all + pd.off;
    float *phiA = phiA_all + pd.off;
    const float4 *prop = prop_all ? prop_all + pd.off : nullptr;
    const int H = P.H, W = P.W, s = lv.s;
    const int ci = item.y, cj = item.z;
    const int x0 = max(0, (ci - 1) * s), x1 = min(W, (ci + 2) * s);
    const int y0 = max(0, (cj - 1) * s), y1 = min(H, (cj + 2) * s);
    const int w = x1 - x0, h = y1 - y0, n = w * h;
    const int cx0 = ci * s, cy0 = cj * s, cw = min(W, cx0 + s) - cx0, chh = min(H, cy0 + s) - cy0;
    int *res = slots + (size_t)ridx * slot_ints;
    const GridSlot gs = grid_slot(res, n);
    int *v = gs.v, *hh = gs.hh, *list = gs.list;
    uint32_t *bits = gs.bits;
    RegionCtx x{sync + ridx, G, c, 0u, &s_flag, &s_val};
    if (threadIdx.x == 0) s_flag = 0;  // read only by thread 0
    const int i0 = grid_range_start(n, c, G), i1 = grid_range_start(n, c + 1, G);
    double rd = 0.5 * (kp.disp_max - kp.disp_min) * ldexp(1.0, -iter);
    double rn = ldexp(1.0, -iter);
    long long acck[4] = {0, 0, 0, 0}, hits = 0;
    CutCount cc{0, 0, 0};
    const int kc = prop ? lv.k_cnn : 0, kr = lv.k_rans;
    const int nprop = lv.k_prop + kr + kc + lv.k_rand;
    const int K = kp.visit;
    const int ntx = (w + kGridTileW - 1) / kGridTileW, nty = (h + kGridTileH - 1) / kGridTileH;
    bool ok = true;
    for (int t0 = 0; t0 < nprop && ok; t0 += K) {
        const int t1 = min(nprop, t0 + K);
        if (c == 0) {
            for (int t = t0; t < t1; ++t) {
                const unsigned long long stream = proposal_stream(kp.seed, iter, level, ci, cj, t);
                if (t >= lv.k_prop && t < lv.k_prop + kr) {
                    // the quantised disparities of a large cell go to the slot (not in use yet)
                    RansacSmem *rsm = reinterpret_cast<RansacSmem *>(smf);
                    long long *dq = cw * chh <= kRansacMaxCell ? rsm->dq : reinterpret_cast<long long *>(res);
                    ransac_cta(lab, W, stream, cx0, cy0, cw, chh, rsm, dq, &s_alpha[t - t0]);
                    continue;
                }
                if (threadIdx.x != 0) continue;
                if (t >= lv.k_prop + kr && t < lv.k_prop + kr + kc) {
                    s_alpha[t - t0] = propose(prop, W, stream, cx0, cy0, cw, chh, false, 0.0, 0.0, 0.0, 0.0);
                    continue;
                }
                const bool perturb = t >= lv.k_prop + kr + kc;
                s_alpha[t - t0] = propose(lab, W, stream, cx0, cy0, cw, chh, perturb, perturb ? rd : 0.0,
                                          perturb ? rn : 0.0, kp.disp_min, kp.disp_max);
                if (perturb) {
                    rd *= 0.5;
                    rn *= 0.5;
                }
            }
            __syncthreads();
            // published by the thread that releases at the barrier
            if (threadIdx.x == 0)
                for (int t = 0; t < t1 - t0; ++t) x.rs->alpha[t] = s_alpha[t];
        }
        if (!(ok = region_sync(x))) break;
        for (int t = t0; t < t1; ++t) {
            const float4 al = __ldcg(&x.rs->alpha[t - t0]);
            // data term phi_p(alpha) on the tiles of the region, into phiA
            for (int q = c; q < ntx * nty; q += G) {
                const int ty = q / ntx, tx = q - ty * ntx;
                const int tx0 = x0 + tx * kGridTileW, ty0 = y0 + ty * kGridTileH;
                const int tw = min(kGridTileW, x1 - tx0), th = min(kGridTileH, y1 - ty0);
                region_unary(P, kp, tx0, ty0, tw, th, al.x, al.y, al.z, smf, phiA + (size_t)ty0 * W + tx0, W);
            }
            if (!(ok = region_sync(x))) break;
            for (int j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
                const int iy = j / w, ix = j - iy * w;
                NodeCaps o;
                build_node(P, kp, lab, al, phiA[(size_t)(y0 + iy) * W + x0 + ix], x0, y0, w, h, ix, iy, o);
                v[j] = o.cap_s - o.cap_t;
                for (int d = 0; d < 4; ++d) res[(size_t)d * n + j] = o.k[d];
                for (int d = 4; d < 8; ++d) res[(size_t)d * n + j] = 0;
            }
            if (!(ok = region_sync(x))) break;
            grid_clamp_terminals(n, w, h, res, v, i0, i1);
            if (!(ok = region_sync(x))) break;
            const int st = grid_maxflow(n, w, h, res, v, hh, list, bits, i0, i1, kp.max_rounds, kp.gr_interval, x,
                                        cc, &s_cnt);
            if (st == LEM_OK) {
                for (int j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
                    if (hh[j] == kGridInf) continue;
                    const int iy = j / w, ix = j - iy * w;
                    const size_t p = (size_t)(y0 + iy) * W + x0 + ix;
                    lab[p] = make_float4(al.x, al.y, al.z, phiA[p]);
                    ++acck[proposal_kind(lv, kc, t)];
                }
            } else {
                ++hits;
                if (st != LEM_ERR_MAXFLOW_LIMIT) {
                    ok = false;
                    break;
                }
            }
            if (!(ok = region_sync(x))) break;
        }
    }
    add_accepted(acck, red, ctr);
    if (threadIdx.x == 0) {
        if (c == 0) {
            // a region whose barriers gave up counts as a cut that did not finish
            atomicAdd(&ctr->limit_hits, (unsigned long long)(hits + (ok ? 0 : 1)));
            atomicAdd(&ctr->evals, (unsigned long long)n * (unsigned long long)nprop);
            atomicAdd(&ctr->rounds, (unsigned long long)cc.rounds);
            atomicAdd(&ctr->relabels, (unsigned long long)cc.relabels);
            atomicAdd(&ctr->bfs_levels, (unsigned long long)cc.levels);
        }
    }
}

// The min-cut of lem_mincut_batch for regions above the shared-memory cut:
// G co-resident CTAs per region, the graph in the region's global slot.
//   flow: zeroed by the caller (each CTA adds its share)
template <int NT>
__global__ void __launch_bounds__(NT, 1)
    k_mincut_grid(KParams kp, const int4 *regions, const int64_t *offsets, int G, const int32_t *tcaps,
                  const int32_t *ncaps, uint8_t *take, int64_t *flow, int32_t *status, int *slots,
                  long long slot_ints, RegionSync *sync, Counters *ctr) {
    __shared__ long long red[33];
    __shared__ int s_flag, s_val, s_cnt;
    const int ridx = blockIdx.x / G, c = blockIdx.x - ridx * G;
    const int4 R = regions[ridx];
    const int w = R.z, h = R.w, n = w * h;
    const int64_t off = offsets[ridx];
    int *res = slots + (size_t)ridx * slot_ints;
    const GridSlot gs = grid_slot(res, n);
    int *v = gs.v, *hh = gs.hh, *list = gs.list;
    uint32_t *bits = gs.bits;
    RegionCtx x{sync + ridx, G, c, 0u, &s_flag, &s_val};
    if (threadIdx.x == 0) s_flag = 0;  // read only by thread 0
    const int i0 = grid_range_start(n, c, G), i1 = grid_range_start(n, c + 1, G);
    for (int j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
        const int iy = j / w, ix = j - iy * w;
        v[j] = tcaps[2 * (off + j)] - tcaps[2 * (off + j) + 1];
        for (int k = 0; k < 8; ++k) {
            int cap = 0;
            const int jx = ix + dir_dx(k), jy = iy + dir_dy(k);
            if (k < 4 && jx >= 0 && jx < w && jy >= 0 && jy < h) cap = max(0, (int)ncaps[4 * (off + j) + k]);
            res[(size_t)k * n + j] = cap;
        }
    }
    int st = LEM_ERR_CUDA;
    CutCount cc{0, 0, 0};
    long long capt = 0;
    if (region_sync(x)) {
        grid_clamp_terminals(n, w, h, res, v, i0, i1);
        if (region_sync(x)) {
            for (int j = i0 + threadIdx.x; j < i1; j += blockDim.x) capt += max(0, -v[j]);
            st = grid_maxflow(n, w, h, res, v, hh, list, bits, i0, i1, kp.max_rounds, kp.gr_interval, x, cc, &s_cnt);
        }
    }
    long long rt = 0;
    for (int j = i0 + threadIdx.x; j < i1; j += blockDim.x) {
        take[off + j] = (st == LEM_OK && hh[j] != kGridInf) ? 1 : 0;
        rt += max(0, -v[j]);
    }
    const long long part = block_sum_ll(capt - rt, red);
    if (threadIdx.x == 0) {
        atomicAdd(reinterpret_cast<unsigned long long *>(&flow[ridx]), (unsigned long long)part);
        if (c == 0) {
            status[ridx] = st;
            atomicAdd(&ctr->rounds, (unsigned long long)cc.rounds);
            atomicAdd(&ctr->relabels, (unsigned long long)cc.relabels);
            atomicAdd(&ctr->bfs_levels, (unsigned long long)cc.levels);
        }
    }
}

size_t unary_bytes_host(const KParams &kp, int H, int W, int rw, int rh) {
    const int r = kp.r, T = kp.T;
    if (kp.bf) {
        const size_t mw = std::min(W, rw + 4 * r), mh = std::min(H, rh + 4 * r);
        return mw * mh * 8;
    }
    const int Mw = std::min(W, rw + 4 * r), Kw = std::min(W, rw + 2 * r);
    (void)rh;
    const int RS = T + 2 * r, RSA = RS + 4;
    return sizeof(float) * ((size_t)RS * 4 * Mw + (size_t)T * 4 * Mw + (size_t)T * 4 * Kw + (size_t)RSA * 4 * Kw);
}

// threads per CTA for a region of n nodes: about 4-8 nodes per thread

cudaError_t set_smem(const void *fn, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

}  // namespace

size_t unary_smem_bytes(const KParams &kp, int H, int W, int rw, int rh) { return unary_bytes_host(kp, H, W, rw, rh); }
size_t cut_smem_bytes(int w, int h) {
    const size_t n = (size_t)w * h;
    const size_t planes = (size_t)11 * h * ((w + 31) / 32) * sizeof(uint32_t);
    const size_t list = ((n + 1) & ~(size_t)1) * sizeof(uint16_t);
    return ((9 * n * sizeof(int) + 15) & ~(size_t)15) + ((n + 1) & ~(size_t)1) * sizeof(uint16_t) +
           std::max(planes, list);
}

cudaError_t launch_preprocess(const uint8_t *left, int64_t lstride, const uint8_t *right, int64_t rstride, int H,
                              int W, float lambda, float eps_w, float gamma, void *Lp, void *Rp, int fmt,
                              float4 *wfw, cudaStream_t st) {
    dim3 grid((W + 127) / 128, H);
    k_preprocess<<<grid, 128, 0, st>>>(left, lstride, right, rstride, H, W, lambda, eps_w, gamma, Lp, Rp, fmt, wfw);
    return cudaGetLastError();
}

cudaError_t launch_guide_stats(const uint8_t *left, int64_t lstride, int H, int W, int r, double eps,
                               double cond_fp64, float4 *gst, int *n_fp64, cudaStream_t st) {
    dim3 grid((W + 127) / 128, H);
    k_guide_stats<<<grid, 128, 0, st>>>(left, lstride, H, W, r, eps, cond_fp64, gst, n_fp64);
    return cudaGetLastError();
}

cudaError_t launch_init_labels(int H, int W, unsigned long long seed, double dmin, double dmax, float4 *lab,
                               cudaStream_t st) {
    dim3 grid((W + 127) / 128, H);
    k_init_labels<<<grid, 128, 0, st>>>(H, W, seed, dmin, dmax, lab);
    return cudaGetLastError();
}

cudaError_t launch_pixel_costs(const DevPlanes &P, const KParams &kp, float4 *lab, int threads, cudaStream_t st) {
    const size_t sm = unary_bytes_host(kp, P.H, P.W, 1, 1);
    cudaError_t e = set_smem((const void *)k_pixel_costs, sm);
    if (e != cudaSuccess) return e;
    k_pixel_costs<<<P.H * P.W, threads, sm, st>>>(P, kp, lab);
    return cudaGetLastError();
}

cudaError_t launch_unary_batch(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                               const int4 *regions, const int64_t *offsets, int n_regions, int K, int max_w,
                               int max_h, const float *labels, float *costs, int threads, cudaStream_t st) {
    const size_t sm = unary_bytes_host(kp, P.H, P.W, max_w, max_h);
    cudaError_t e = set_smem((const void *)k_unary_batch, sm);
    if (e != cudaSuccess) return e;
    k_unary_batch<<<n_regions * K, threads, sm, st>>>(P, kp, pairs, img, regions, offsets, K, labels, costs);
    return cudaGetLastError();
}

cudaError_t launch_pairwise_batch(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                                  const int4 *regions, const int64_t *offsets, int n_regions, const float4 *lab,
                                  const float *alpha, const float *costs_alpha, int32_t *tcaps, int32_t *ncaps,
                                  int64_t *cterm, int threads, cudaStream_t st) {
    k_pairwise_batch<<<n_regions, threads, 0, st>>>(P, kp, pairs, img, regions, offsets, lab, alpha, costs_alpha,
                                                    tcaps, ncaps, cterm);
    return cudaGetLastError();
}

template <int NT>
cudaError_t mincut_nt(const KParams &kp, const int4 *regions, const int64_t *offsets, int n_regions, size_t sm,
                      const int32_t *tcaps, const int32_t *ncaps, uint8_t *take, int64_t *flow, int32_t *status,
                      Counters *ctr, cudaStream_t st) {
    cudaError_t e = set_smem((const void *)k_mincut_batch<NT>, sm);
    if (e != cudaSuccess) return e;
    k_mincut_batch<NT><<<n_regions, NT, sm, st>>>(kp, regions, offsets, tcaps, ncaps, take, flow, status, ctr);
    return cudaGetLastError();
}

cudaError_t launch_mincut_batch(const KParams &kp, const int4 *regions, const int64_t *offsets, int n_regions,
                                int max_nodes, size_t smem, const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                                int64_t *flow, int32_t *status, Counters *ctr, cudaStream_t st) {
    const size_t sm = smem;
    const int nt = threads_for_nodes(max_nodes);
    if (nt == 256) return mincut_nt<256>(kp, regions, offsets, n_regions, sm, tcaps, ncaps, take, flow, status, ctr, st);
    if (nt == 512) return mincut_nt<512>(kp, regions, offsets, n_regions, sm, tcaps, ncaps, take, flow, status, ctr, st);
    return mincut_nt<1024>(kp, regions, offsets, n_regions, sm, tcaps, ncaps, take, flow, status, ctr, st);
}

template <int NT>
cudaError_t expand_nt(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter, const int *iter_dev,
                      const PairDesc *pairs, const int4 *items, int n_items, float4 *lab, float *phiA,
                      const float4 *prop, Counters *ctr, float *phiB, int *queue, unsigned *done, size_t sm,
                      cudaStream_t st) {
    cudaError_t e;
    if (!phiB) {
        if ((e = set_smem((const void *)k_expand_group<NT, false>, sm)) != cudaSuccess) return e;
        int grid = n_items;
        if (queue) {
            // work queue: at most as many CTAs as are co-resident
            int per_sm = 0, dev = 0, nsm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_group<NT, false>, NT, sm) !=
                    cudaSuccess ||
                cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();
                per_sm = 1;
                nsm = 1;
            }
            grid = std::max(1, std::min(n_items, per_sm * nsm));
        }
        k_expand_group<NT, false><<<grid, NT, sm, st>>>(P, kp, lv, level, iter, iter_dev, pairs, items, lab, phiA,
                                                        prop, ctr, nullptr, n_items, queue, done);
        return cudaGetLastError();
    }
    if ((e = set_smem((const void *)k_expand_group<NT, true>, sm)) != cudaSuccess) return e;
    // two CTAs per region, co-scheduled as a cluster
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * n_items);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // The second CTA only pays off on SMs the launch would leave idle: with more
    // regions than one wave of single CTAs holds, or on a device that cannot
    // co-schedule the pair, one CTA per region (same result).
    int clusters = 0, per_sm = 0, dev = 0, nsm = 0;
    const bool ok = cudaOccupancyMaxActiveClusters(&clusters, k_expand_group<NT, true>, &cfg) == cudaSuccess &&
                    cudaGetDevice(&dev) == cudaSuccess &&
                    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_group<NT, true>, NT, sm) ==
                        cudaSuccess;
    if (!ok || clusters < n_items || 2 * n_items > per_sm * nsm) {
        cudaGetLastError();
        return expand_nt<NT>(P, kp, lv, level, iter, iter_dev, pairs, items, n_items, lab, phiA, prop, ctr, nullptr,
                             queue, nullptr, sm, st);
    }
    return cudaLaunchKernelEx(&cfg, k_expand_group<NT, true>, P, kp, lv, level, iter, iter_dev, pairs, items, lab,
                              phiA, prop, ctr, phiB, n_items, (int *)nullptr, (unsigned *)nullptr);
}

cudaError_t launch_expand_group(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                                const int *iter_dev, const PairDesc *pairs, int max_w, int max_h, const int4 *items,
                                int n_items, float4 *lab, float *phiA, const float4 *prop, Counters *ctr, float *phiB,
                                int *queue, unsigned *done, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    if (done && !queue) return cudaErrorInvalidValue;
    const int s = lv.s;
    const int rw = std::min(max_w, 3 * s), rh = std::min(max_h, 3 * s);
    size_t sm = std::max(unary_bytes_host(kp, max_h, max_w, rw, rh), cut_smem_bytes(rw, rh));
    if (lv.k_rans > 0) sm = std::max(sm, sizeof(RansacSmem));
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    const int nt = lv.threads > 0 ? lv.threads : threads_for_nodes(rw * rh);
    if (nt != 128 && nt != 256 && nt != 512 && nt != 1024) return cudaErrorInvalidValue;
    // the two-CTA visit only for two propagation candidates per visit
    const bool two = !done && phiB && lv.k_prop == 2 && lv.k_rand == 0 && lv.k_rans == 0 && (lv.k_cnn == 0 || !prop);
    float *pb = two ? phiB : nullptr;
#define LEM_EXPAND_NT(NT_) \
    expand_nt<NT_>(P, kp, lv, level, iter, iter_dev, pairs, items, n_items, lab, phiA, prop, ctr, pb, queue, done, sm, \
                   st)
    if (nt == 128) return LEM_EXPAND_NT(128);
    if (nt == 256) return LEM_EXPAND_NT(256);
    if (nt == 512) return LEM_EXPAND_NT(512);
    return LEM_EXPAND_NT(1024);
#undef LEM_EXPAND_NT
}

namespace {
// filtering-region width and per-warp ring bytes of the warp data term at a level
struct VisitShape {
    int rw, rh, nc, mwp, kwp;
    size_t ring_bytes;
    int warps;  // most warps (units) per CTA of k_visit_unary
};
VisitShape visit_shape(const KParams &kp, const Level &lv, int max_w, int max_h) {
    VisitShape v;
    v.rw = std::min(max_w, 3 * lv.s);
    v.rh = std::min(max_h, 3 * lv.s);
    v.mwp = std::min(max_w, v.rw + 4 * kp.r);
    v.kwp = std::min(max_w, v.rw + 2 * kp.r);
    v.nc = (v.mwp + 31) / 32;
    v.ring_bytes = sizeof(float) * (size_t)warp_ring_floats(kp.r, v.mwp, v.kwp);
    v.warps = (int)std::min<size_t>(4, (227 * 1024) / v.ring_bytes);
    return v;
}

// warps per CTA of a warp data-term launch of `units` units: up to `most` (the
// shared-memory limit), fewer when the launch would not give every SM two CTAs
int warps_per_cta(int units, int most) {
    int dev = 0, nsm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        nsm = 152;
    }
    int w = std::max(1, std::min(4, most));
    while (w > 1 && (units + w - 1) / w < 2 * nsm) w >>= 1;
    return w;
}

template <int NC>
cudaError_t unary_batch_warp_nc(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                                const int4 *regions, const int64_t *offsets, int n_regions, int K,
                                const float *labels, float *costs, int mwp, int kwp, int most, cudaStream_t st) {
    const size_t ring = sizeof(float) * (size_t)warp_ring_floats(kp.r, mwp, kwp);
    const int units = n_regions * K, w = warps_per_cta(units, most);
    cudaError_t e = set_smem((const void *)k_unary_batch_warp<NC>, ring * w);
    if (e != cudaSuccess) return e;
    k_unary_batch_warp<NC><<<(units + w - 1) / w, 32 * w, ring * w, st>>>(P, kp, pairs, img, regions, offsets,
                                                                          n_regions, K, labels, costs, mwp, kwp);
    return cudaGetLastError();
}

template <int NC>
cudaError_t visit_unary_nc(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                           const int *iter_dev, const PairDesc *pairs, const int4 *items, int n_items, int t0, int nK,
                           const float4 *lab, float *phiK, long long plane_stride, const float4 *prop, float4 *alphaK,
                           int mwp, int kwp, int most, cudaStream_t st) {
    const size_t ring = sizeof(float) * (size_t)warp_ring_floats(kp.r, mwp, kwp);
    const int units = n_items * nK, w = warps_per_cta(units, most);
    cudaError_t e = set_smem((const void *)k_visit_unary<NC>, ring * w);
    if (e != cudaSuccess) return e;
    k_visit_unary<NC><<<(units + w - 1) / w, 32 * w, ring * w, st>>>(
        P, kp, lv, level, iter, iter_dev, pairs, items, n_items, t0, nK, lab, phiK, plane_stride, prop, alphaK, mwp,
        kwp);
    return cudaGetLastError();
}

template <int NT>
cudaError_t visit_cut_nt(const DevPlanes &P, const KParams &kp, const Level &lv, const PairDesc *pairs,
                         const int4 *items, int n_items, int t0, int nK, int kc, float4 *lab, const float *phiK,
                         long long plane_stride, const float4 *alphaK, Counters *ctr, size_t smem, cudaStream_t st) {
    cudaError_t e = set_smem((const void *)k_visit_cut<NT>, smem);
    if (e != cudaSuccess) return e;
    k_visit_cut<NT><<<n_items, NT, smem, st>>>(P, kp, lv, pairs, items, t0, nK, kc, lab, phiK, plane_stride, alphaK,
                                               ctr);
    return cudaGetLastError();
}
}  // namespace

bool visit_split(const KParams &kp, const Level &lv, int max_w, int max_h) {
    if (kp.visit < 2 || kp.bf || lv.k_rans > 0) return false;
    const VisitShape v = visit_shape(kp, lv, max_w, max_h);
    if ((long long)v.rw * v.rh > LEM_MAX_REGION_NODES || cut_smem_bytes(v.rw, v.rh) > 227 * 1024) return false;
    return v.nc <= 4 && v.warps >= 1;
}

bool unary_warp_fits(const KParams &kp, int W, int max_w) {
    const int mwp = std::min(W, max_w + 4 * kp.r), kwp = std::min(W, max_w + 2 * kp.r);
    return !kp.bf && (mwp + 31) / 32 <= 4 && sizeof(float) * (size_t)warp_ring_floats(kp.r, mwp, kwp) <= 227 * 1024;
}

cudaError_t launch_unary_batch_warp(const DevPlanes &P, const KParams &kp, const PairDesc *pairs, const int *img,
                                    const int4 *regions, const int64_t *offsets, int n_regions, int K, int max_w,
                                    const float *labels, float *costs, cudaStream_t st) {
    const int mwp = std::min(P.W, max_w + 4 * kp.r), kwp = std::min(P.W, max_w + 2 * kp.r);
    const int nc = (mwp + 31) / 32;
    const int most =
        (int)std::min<size_t>(4, (227 * 1024) / (sizeof(float) * (size_t)warp_ring_floats(kp.r, mwp, kwp)));
#define LEM_UBW(NC_) \
    unary_batch_warp_nc<NC_>(P, kp, pairs, img, regions, offsets, n_regions, K, labels, costs, mwp, kwp, most, st)
    switch (nc) {
        case 1: return LEM_UBW(1);
        case 2: return LEM_UBW(2);
        case 3: return LEM_UBW(3);
        case 4: return LEM_UBW(4);
        default: return cudaErrorInvalidConfiguration;
    }
#undef LEM_UBW
}

int visit_cut_threads(int nodes) { return nodes <= 400 ? 64 : (nodes <= 2500 ? 256 : 512); }

cudaError_t launch_visit_unary(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                               const int *iter_dev, const PairDesc *pairs, int max_w, int max_h, const int4 *items,
                               int n_items, int t0, int nK, const float4 *lab, float *phiK, long long plane_stride,
                               const float4 *prop, float4 *alphaK, cudaStream_t st) {
    if (n_items == 0 || nK < 1) return cudaSuccess;
    const VisitShape v = visit_shape(kp, lv, max_w, max_h);
#define LEM_VISIT_UNARY(NC_)                                                                                      \
    visit_unary_nc<NC_>(P, kp, lv, level, iter, iter_dev, pairs, items, n_items, t0, nK, lab, phiK, plane_stride, \
                        prop, alphaK, v.mwp, v.kwp, v.warps, st)
    switch (v.nc) {
        case 1: return LEM_VISIT_UNARY(1);
        case 2: return LEM_VISIT_UNARY(2);
        case 3: return LEM_VISIT_UNARY(3);
        case 4: return LEM_VISIT_UNARY(4);
        default: return cudaErrorInvalidConfiguration;
    }
#undef LEM_VISIT_UNARY
}

cudaError_t launch_visit_cut(const DevPlanes &P, const KParams &kp, const Level &lv, const PairDesc *pairs,
                             int max_w, int max_h, const int4 *items, int n_items, int t0, int nK, int kc,
                             float4 *lab, const float *phiK, long long plane_stride, const float4 *alphaK,
                             Counters *ctr, cudaStream_t st) {
    if (n_items == 0 || nK < 1) return cudaSuccess;
    const VisitShape v = visit_shape(kp, lv, max_w, max_h);
    const size_t csm = cut_smem_bytes(v.rw, v.rh);
    const int nt = lv.threads > 0 ? lv.threads : visit_cut_threads(v.rw * v.rh);
#define LEM_VISIT_CUT(NT_) \
    visit_cut_nt<NT_>(P, kp, lv, pairs, items, n_items, t0, nK, kc, lab, phiK, plane_stride, alphaK, ctr, csm, st)
    switch (nt) {
        case 32: return LEM_VISIT_CUT(32);
        case 64: return LEM_VISIT_CUT(64);
        case 128: return LEM_VISIT_CUT(128);
        case 256: return LEM_VISIT_CUT(256);
        case 512: return LEM_VISIT_CUT(512);
        case 1024: return LEM_VISIT_CUT(1024);
        default: return cudaErrorInvalidValue;
    }
#undef LEM_VISIT_CUT
}

bool expand_uses_grid(const KParams &kp, const Level &lv, int max_w, int max_h) {
    const int s = lv.s;
    const int rw = std::min(max_w, 3 * s), rh = std::min(max_h, 3 * s);
    if ((long long)rw * rh > LEM_MAX_REGION_NODES) return true;
    size_t sm = std::max(unary_bytes_host(kp, max_h, max_w, rw, rh), cut_smem_bytes(rw, rh));
    if (lv.k_rans > 0) sm = std::max(sm, sizeof(RansacSmem));
    return sm > 227 * 1024;
}

long long grid_slot_ints_host(int max_w, int max_h, int s) {
    return grid_slot_ints(std::min(max_w, 3 * s), std::min(max_h, 3 * s));
}

size_t grid_sync_bytes() { return sizeof(RegionSync); }

long long grid_slot_ints_wh(int w, int h) { return grid_slot_ints(w, h); }

cudaError_t launch_expand_grid(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                               const PairDesc *pairs, int max_w, int max_h, const int4 *items, int n_items,
                               float4 *lab, float *phiA, const float4 *prop, Counters *ctr, int *slots,
                               long long slot_cap_ints, void *sync, int sync_cap, cudaStream_t st) {
    if (n_items == 0) return cudaSuccess;
    const int s = lv.s;
    const int rw = std::min(max_w, 3 * s), rh = std::min(max_h, 3 * s);
    size_t sm = unary_bytes_host(kp, max_h, max_w, std::min(rw, kGridTileW), std::min(rh, kGridTileH));
    if (lv.k_rans > 0) sm = std::max(sm, sizeof(RansacSmem));
    if (sm > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = set_smem((const void *)k_expand_grid<kGridThreads>, sm);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expand_grid<kGridThreads>, kGridThreads,
                                                           sm)) != cudaSuccess)
        return e;
    const int cap = per_sm * nsm;
    const long long slot_ints = grid_slot_ints(rw, rh);
    const long long by_slots = slot_cap_ints / slot_ints;
    const int chunk = (int)std::min<long long>({(long long)n_items, (long long)cap, (long long)sync_cap, by_slots});
    if (chunk < 1) return cudaErrorInvalidConfiguration;
    const int nodes = rw * rh;
    for (int b = 0; b < n_items; b += chunk) {
        const int m = std::min(chunk, n_items - b);
        // CTAs per region: all co-resident, and at least 2048 nodes each
        int G = std::max(1, std::min(cap / m, (nodes + 2047) / 2048));
        if ((e = cudaMemsetAsync(sync, 0, sizeof(RegionSync) * m, st)) != cudaSuccess) return e;
        DevPlanes Pc = P;
        KParams kc = kp;
        Level lc = lv;
        int lvl = level, it = iter, g = G;
        const PairDesc *pp = pairs;
        const int4 *ip = items + b;
        float4 *lp = lab;
        float *fp = phiA;
        const float4 *prp = prop;
        int *sp = slots;
        long long si = slot_ints;
        RegionSync *syp = reinterpret_cast<RegionSync *>(sync);
        Counters *cp = ctr;
        void *args[] = {&Pc, &kc, &lc, &lvl, &it, &g, &pp, &ip, &lp, &fp, &prp, &sp, &si, &syp, &cp};
        e = cudaLaunchCooperativeKernel((const void *)k_expand_grid<kGridThreads>, dim3(m * G), dim3(kGridThreads),
                                        args, sm, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_mincut_grid(const KParams &kp, const int4 *regions, const int64_t *offsets, int n_regions,
                               int max_w, int max_h, const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                               int64_t *flow, int32_t *status, Counters *ctr, int *slots, long long slot_cap_ints,
                               void *sync, int sync_cap, cudaStream_t st) {
    int per_sm = 0, dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mincut_grid<kGridThreads>, kGridThreads, 0)) !=
        cudaSuccess)
        return e;
    const int cap = per_sm * nsm;
    const long long slot_ints = grid_slot_ints(max_w, max_h);
    const int chunk = (int)std::min<long long>(
        {(long long)n_regions, (long long)cap, (long long)sync_cap, slot_cap_ints / slot_ints});
    if (chunk < 1) return cudaErrorInvalidConfiguration;
    if ((e = cudaMemsetAsync(flow, 0, sizeof(int64_t) * n_regions, st)) != cudaSuccess) return e;
    const int nodes = max_w * max_h;
    for (int b = 0; b < n_regions; b += chunk) {
        const int m = std::min(chunk, n_regions - b);
        int G = std::max(1, std::min(cap / m, (nodes + 2047) / 2048));
        if ((e = cudaMemsetAsync(sync, 0, sizeof(RegionSync) * m, st)) != cudaSuccess) return e;
        KParams kc = kp;
        const int4 *rp = regions + b;
        const int64_t *op = offsets + b;
        int g = G;
        const int32_t *tp = tcaps, *np = ncaps;
        uint8_t *tk = take;
        int64_t *fp = flow + b;
        int32_t *sp = status + b;
        int *sl = slots;
        long long si = slot_ints;
        RegionSync *syp = reinterpret_cast<RegionSync *>(sync);
        Counters *cp = ctr;
        void *args[] = {&kc, &rp, &op, &g, &tp, &np, &tk, &fp, &sp, &sl, &si, &syp, &cp};
        e = cudaLaunchCooperativeKernel((const void *)k_mincut_grid<kGridThreads>, dim3(m * G), dim3(kGridThreads),
                                        args, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void k_increment(int *x) { *x += 1; }

cudaError_t launch_propose_batch(const DevPlanes &P, const KParams &kp, const Level &lv, int level, int iter,
                                 const int2 *cells, int n_cells, const float4 *lab, const float4 *prop, float *alpha,
                                 long long *dq_scratch, cudaStream_t st) {
    if (n_cells == 0) return cudaSuccess;
    if (lv.k_rans > 0 && lv.s * lv.s > kRansacMaxCell && !dq_scratch) return cudaErrorInvalidValue;
    const size_t sm = sizeof(RansacSmem);
    cudaError_t e = set_smem((const void *)k_propose_batch, sm);
    if (e != cudaSuccess) return e;
    k_propose_batch<<<n_cells, 128, sm, st>>>(P, kp, lv, level, iter, cells, lab, prop, alpha,
                                              lv.s * lv.s > kRansacMaxCell ? dq_scratch : nullptr);
    return cudaGetLastError();
}

cudaError_t launch_increment(int *x, cudaStream_t st) {
    k_increment<<<1, 1, 0, st>>>(x);
    return cudaGetLastError();
}

int energy_partials(int H, int W) { return std::min(1024, (H * W + 255) / 256); }

cudaError_t launch_cnn_features(const DevPlanes &P, const float4 *lab, float dmax, float *x, cudaStream_t st) {
    const int H4 = (P.H + 3) / 4, W4 = (P.W + 3) / 4;
    k_cnn_features<<<(H4 * W4 + 255) / 256, 256, 0, st>>>(P, lab, H4, W4, 1.f / dmax, x);
    return cudaGetLastError();
}
cudaError_t launch_cnn_targets(const float4 *lab, int H, int W, float dmax, float *t, cudaStream_t st) {
    const int H4 = (H + 3) / 4, W4 = (W + 3) / 4;
    k_cnn_targets<<<(H4 * W4 + 255) / 256, 256, 0, st>>>(lab, H, W, H4, W4, 1.f / dmax, t);
    return cudaGetLastError();
}
cudaError_t launch_cnn_upsample(const float *y, int H, int W, float dmax, float4 *prop, cudaStream_t st) {
    const int H4 = (H + 3) / 4, W4 = (W + 3) / 4;
    k_cnn_upsample<<<(H * W + 255) / 256, 256, 0, st>>>(y, H4, W4, H, W, dmax, prop);
    return cudaGetLastError();
}
cudaError_t launch_props_in(int n, const float *abc, float4 *prop, cudaStream_t st) {
    k_props_in<<<(n + 255) / 256, 256, 0, st>>>(n, abc, prop);
    return cudaGetLastError();
}
cudaError_t launch_props_out(int n, const float4 *prop, float *abc, cudaStream_t st) {
    k_props_out<<<(n + 255) / 256, 256, 0, st>>>(n, prop, abc);
    return cudaGetLastError();
}

// Packed 8-bit RGB from an image of any element type and layout: the first
// three values of each pixel, a float rounded to the nearest integer and
// clamped to [0, 255] (NaN to 0).
__global__ void k_to_rgb8(const unsigned char *src, int64_t srow, int64_t spx, int dtype, int H, int W,
                          uint8_t *dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const unsigned char *s = src + (size_t)y * srow + (size_t)x * spx;
    uint8_t *d = dst + ((size_t)y * W + x) * 3;
    for (int c = 0; c < 3; ++c) {
        if (dtype == LEM_IMG_U8) {
            d[c] = s[c];
            continue;
        }
        float v;
        if (dtype == LEM_IMG_F16) v = __half2float(reinterpret_cast<const __half *>(s)[c]);
        else if (dtype == LEM_IMG_BF16) v = __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(s)[c]);
        else v = reinterpret_cast<const float *>(s)[c];
        d[c] = (uint8_t)rintf(fminf(fmaxf(v, 0.f), 255.f));
    }
}

cudaError_t launch_to_rgb8(const void *src, int64_t srow, int64_t spx, int dtype, int H, int W, uint8_t *dst,
                           cudaStream_t st) {
    dim3 grid((W + 255) / 256, H);
    k_to_rgb8<<<grid, 256, 0, st>>>((const unsigned char *)src, srow, spx, dtype, H, W, dst);
    return cudaGetLastError();
}

__global__ void k_mirror_rgb(const uint8_t *src, int64_t stride, int H, int W, uint8_t *dst) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= W || y >= H) return;
    const uint8_t *s = src + (size_t)y * stride + 3 * (size_t)(W - 1 - x);
    uint8_t *d = dst + ((size_t)y * W + x) * 3;
    d[0] = s[0];
    d[1] = s[1];
    d[2] = s[2];
}

cudaError_t launch_mirror_rgb(const uint8_t *src, int64_t stride, int H, int W, uint8_t *dst, cudaStream_t st) {
    dim3 grid((W + 255) / 256, H);
    k_mirror_rgb<<<grid, 256, 0, st>>>(src, stride, H, W, dst);
    return cudaGetLastError();
}

cudaError_t launch_postprocess(const DevPlanes &PL, const float4 *labL, const float4 *labRm, float thr, int radius,
                               float gamma, uint8_t *valid, float *filled, float *disp, cudaStream_t st) {
    const int n = PL.H * PL.W;
    k_lr_check<<<(n + 255) / 256, 256, 0, st>>>(labL, labRm, PL.H, PL.W, thr, valid);
    k_fill<<<(n + 255) / 256, 256, 0, st>>>(labL, valid, PL.H, PL.W, filled);
    const long long threads = 32LL * n;
    k_wmedian<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(PL, valid, filled, radius, 1.0f / gamma, disp);
    return cudaGetLastError();
}

cudaError_t launch_energy(const DevPlanes &P, const KParams &kp, const float4 *lab, long long *partials,
                          long long *out, cudaStream_t st) {
    const int nb = energy_partials(P.H, P.W);
    k_energy<<<nb, 256, 0, st>>>(P, kp, lab, partials);
    k_sum_partials<<<1, 256, 0, st>>>(partials, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_labels_out(int H, int W, const float4 *lab, float *abc, float *disp, float *cost,
                              cudaStream_t st) {
    k_labels_out<<<(H * W + 255) / 256, 256, 0, st>>>(H, W, lab, abc, disp, cost);
    return cudaGetLastError();
}

cudaError_t launch_labels_in(int H, int W, const float *abc, const float *cost, float4 *lab, cudaStream_t st) {
    k_labels_in<<<(H * W + 255) / 256, 256, 0, st>>>(H, W, abc, cost, lab);
    return cudaGetLastError();
}

cudaError_t launch_planes_out(int H, int W, const DevPlanes &P, float *left, float *right, float *guide,
                              float *weights, cudaStream_t st) {
    k_planes_out<<<(H * W + 255) / 256, 256, 0, st>>>(H, W, P, left, right, guide, weights);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Min-cut without allocation.  Some callers cannot allocate device memory at
// the point where they cut (code running inside a preallocated memory arena,
// a host thread that must not call cudaMalloc because it would synchronise
// the device, or an embedding that forbids growing the device heap).  For
// them the per-call scratch of the batch min-cut (region descriptors, their
// packed offsets and the work counters) lives in this fixed array, which every
// GPU that loads the library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocRegionsOff = 0;
constexpr size_t kNoAllocOffsetsOff = kNoAllocRegionsOff + sizeof(int4) * LEM_NOALLOC_MAX_REGIONS;
constexpr size_t kNoAllocCountersOff = kNoAllocOffsetsOff + sizeof(int64_t) * LEM_NOALLOC_MAX_REGIONS;
constexpr size_t kNoAllocBytes = kNoAllocCountersOff + sizeof(Counters);
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// packed offsets of the regions (exclusive prefix sum of w*h), one CTA
__global__ void k_noalloc_offsets(const int4 *regions, int n, int64_t *offsets) {
    __shared__ long long carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const long long sz = i < n ? (long long)regions[i].z * regions[i].w : 0;
        // inclusive scan of sz over the block (Hillis-Steele in shared memory)
        __shared__ long long scan[1024];
        scan[threadIdx.x] = sz;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            const long long add = threadIdx.x >= (unsigned)o ? scan[threadIdx.x - o] : 0;
            __syncthreads();
            scan[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) offsets[i] = carry + scan[threadIdx.x] - sz;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += scan[threadIdx.x];
        __syncthreads();
    }
}

// device address of g_noalloc_scratch per device, taken once per device with
// that device current
struct NoAllocSlot {
    int ready;
    unsigned char *ptr;
};
NoAllocSlot g_noalloc_slots[64];
}  // namespace

cudaError_t noalloc_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    NoAllocSlot &slot = g_noalloc_slots[dev];
    if (!__atomic_load_n(&slot.ready, __ATOMIC_ACQUIRE)) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        slot.ptr = (unsigned char *)p;
        __atomic_store_n(&slot.ready, 1, __ATOMIC_RELEASE);
    }
    *out = slot.ptr;
    return cudaSuccess;
}

cudaError_t launch_mincut_noalloc(const KParams &kp, const lem_region *regions, int n_regions, int max_nodes,
                                  size_t smem, const int32_t *tcaps, const int32_t *ncaps, uint8_t *take,
                                  int64_t *flow, int32_t *status, cudaStream_t st) {
    unsigned char *scr = nullptr;
    cudaError_t e = noalloc_scratch(&scr);
    if (e != cudaSuccess) return e;
    int4 *d_regions = (int4 *)(scr + kNoAllocRegionsOff);
    int64_t *d_offsets = (int64_t *)(scr + kNoAllocOffsetsOff);
    Counters *d_ctr = (Counters *)(scr + kNoAllocCountersOff);
    // the first four ints of each lem_region (x0, y0, w, h), packed as int4
    static_assert(sizeof(lem_region) >= sizeof(int4) && offsetof(lem_region, h) == 3 * sizeof(int),
                  "lem_region starts with x0, y0, w, h");
    e = cudaMemcpy2DAsync(d_regions, sizeof(int4), regions, sizeof(lem_region), sizeof(int4), n_regions,
                          cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d_ctr, 0, sizeof(Counters), st);
    if (e != cudaSuccess) return e;
    k_noalloc_offsets<<<1, 1024, 0, st>>>(d_regions, n_regions, d_offsets);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_mincut_batch(kp, d_regions, d_offsets, n_regions, max_nodes, smem, tcaps, ncaps, take, flow,
                               status, d_ctr, st);
}
}  // namespace lem
