// mpm_device.cuh -- device-side building blocks of the MLS-MPM substep (FP32, sm_103a).
//
// The paper (Sec. 3; App. D.1, Algorithm 1) names the solver, MLS-MPM in the
// style of PlasticineLab, and the order of a soft step; the equations are the
// published methods it points to: quadratic B-spline APIC/MLS transfers
// (Jiang et al. 2015; Hu et al. 2018), fixed-corotated elasticity, von Mises
// plasticity in Hencky strain, a J-only weakly compressible fluid, and
// grid-node Coulomb contact against analytic box / capsule distances.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mpm {

// Grid blocks are 4^3 nodes stored contiguously (block-major): node (i,j,k) lives at
// block ((i>>2)*nb + (j>>2))*nb + (k>>2), slot ((i&3)*4 + (j&3))*4 + (k&3).
constexpr int kBlk = 4;
constexpr int kBlkNodes = 64;
constexpr int kGatherEdge = 6;   // a block's particles read nodes [4b, 4b+6) per axis
constexpr int kScatterEdge = 8;  // after one substep they write nodes [4b-1, 4b+7) per axis
constexpr int kGatherNodes = kGatherEdge * kGatherEdge * kGatherEdge;
constexpr int kScatterNodes = kScatterEdge * kScatterEdge * kScatterEdge;
constexpr int kMaxColliders = 32;

__host__ __device__ __forceinline__ uint32_t block_index(int bx, int by, int bz, int nb) {
    return (uint32_t)((bx * nb + by) * nb + bz);
}

__host__ __device__ __forceinline__ uint32_t node_index(int i, int j, int k, int nb) {
    return block_index(i >> 2, j >> 2, k >> 2, nb) * kBlkNodes + (uint32_t)(((i & 3) * 4 + (j & 3)) * 4 + (k & 3));
}

// Lowest stencil node per axis: floor(x/dx - 0.5). Written with _rn intrinsics so the key pass and
// the transfer passes, in different kernels, always round identically (no FMA contraction).
__device__ __forceinline__ int cell_base(float x, float inv_dx) {
    return __float2int_rd(__fsub_rn(__fmul_rn(x, inv_dx), 0.5f));
}

__device__ __forceinline__ float cell_frac(float x, float inv_dx, int base) {
    return __fsub_rn(__fmul_rn(x, inv_dx), (float)base);
}

// Quadratic B-spline weights of the nodes base, base+1, base+2 at distances fx, fx-1, fx-2 (cells).
__device__ __forceinline__ void bspline_weights(float fx, float w[3]) {
    float a = 1.5f - fx, b = fx - 1.0f, c = fx - 0.5f;
    w[0] = 0.5f * a * a;
    w[1] = 0.75f - b * b;
    w[2] = 0.5f * c * c;
}

// ------------------------------------------------------------------------ polar data of F (FP32)
//
// Everything the constitutive update needs from F = U diag(sig) V^T is U and sig: with the symmetric
// B = F F^T = U diag(sig^2) U^T,
//   (F - R) F^T = U diag((sig - 1) sig) U^T            (R = U V^T, the polar rotation)
//   U diag(s') V^T = U diag(s' / sig) U^T F            (F with its singular values replaced)
// so V is never formed. U and sig^2 come from cyclic Jacobi on B (exact Givens rotations, Golub & Van
// Loan Sec. 8.5.2). sig_i = sqrt(eigenvalue_i) >= 0; when det F < 0 the smallest one takes the sign
// (the rotation-only SVD convention: det U = det V = +1).

template <int P, int Q, int R>
__device__ __forceinline__ void jacobi_rotation(float (&S)[3][3], float (&U)[3][3]) {
    const float apq = S[P][Q];
    if (apq == 0.0f) return;
    // The rotation J (J_pp = J_qq = c, J_pq = s, J_qp = -s) zeroes the (p,q) entry of J^T S J when
    // tan 2theta = 2 a_pq / (a_qq - a_pp). Take |theta| <= pi/4: cos 2theta = |x| / r,
    // sin 2theta = sign(x) y / r with x = a_qq - a_pp, y = 2 a_pq, r = |(x, y)|; then the half angle
    // c = sqrt((1 + cos 2theta) / 2), s = sin 2theta / (2 c). Two reciprocal square roots in all.
    const float app = S[P][P], aqq = S[Q][Q];
    const float x = aqq - app, y = 2.0f * apq;
    const float h = rsqrtf(fmaf(x, x, y * y));
    const float c2 = fabsf(x) * h;
    const float s2 = copysignf(1.0f, x) * y * h;
    const float half = fmaf(0.5f, c2, 0.5f);
    const float rc = rsqrtf(half);
    const float c = half * rc;
    const float s = 0.5f * s2 * rc;
    const float2 sq = __fmul2_rn(make_float2(c, s), make_float2(c, s));  // (c^2, s^2)
    const float cs2 = 2.0f * c * s * apq;
    const float2 dg = __ffma2_rn(sq, make_float2(app, app),
                                 __ffma2_rn(make_float2(sq.y, sq.x), make_float2(aqq, aqq), make_float2(-cs2, cs2)));
    S[P][P] = dg.x;
    S[Q][Q] = dg.y;
    S[P][Q] = S[Q][P] = 0.0f;
    // rows (p, q) of the rotation as packed FP32x2 pairs: (c, s) a_p + (-s, c) a_q
    const float2 cs = make_float2(c, s), nsc = make_float2(-s, c);
    const float arp = S[R][P], arq = S[R][Q];
    const float2 sr = __ffma2_rn(nsc, make_float2(arq, arq), __fmul2_rn(cs, make_float2(arp, arp)));
    S[R][P] = S[P][R] = sr.x;
    S[R][Q] = S[Q][R] = sr.y;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float up = U[r][P], uq = U[r][Q];
        const float2 ur = __ffma2_rn(nsc, make_float2(uq, uq), __fmul2_rn(cs, make_float2(up, up)));
        U[r][P] = ur.x;
        U[r][Q] = ur.y;
    }
}

__device__ __forceinline__ float det3(const float (&A)[3][3]) {
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
           A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// U (left singular vectors, columns) and the signed singular values of F.
__device__ __forceinline__ void polar_data(const float (&F)[3][3], float (&U)[3][3], float (&sig)[3]) {
    float S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            const float b = F[i][0] * F[j][0] + F[i][1] * F[j][1] + F[i][2] * F[j][2];
            S[i][j] = b;
            S[j][i] = b;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) U[i][j] = (i == j) ? 1.0f : 0.0f;
    for (int sweep = 0; sweep < 6; ++sweep) {
        const float off = S[0][1] * S[0][1] + S[0][2] * S[0][2] + S[1][2] * S[1][2];
        const float diag = S[0][0] * S[0][0] + S[1][1] * S[1][1] + S[2][2] * S[2][2];
        if (off <= 1e-13f * diag) break;
        jacobi_rotation<0, 1, 2>(S, U);
        jacobi_rotation<0, 2, 1>(S, U);
        jacobi_rotation<1, 2, 0>(S, U);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) sig[i] = sqrtf(fmaxf(S[i][i], 0.0f));
    if (det3(F) < 0.0f) {  // negate the smallest (first on ties), by selects
        const bool k0 = sig[0] <= sig[1] && sig[0] <= sig[2];
        const bool k1 = !k0 && sig[1] <= sig[2];
        const bool k2 = !k0 && !k1;
        sig[0] = k0 ? -sig[0] : sig[0];
        sig[1] = k1 ? -sig[1] : sig[1];
        sig[2] = k2 ? -sig[2] : sig[2];
    }
}

// U diag(d) U^T (symmetric): rows of U d against pairs of rows of U, as packed FP32x2 products
__device__ __forceinline__ void sym_from_eig(const float (&U)[3][3], const float (&d)[3], float (&M)[3][3]) {
    float Ud[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) Ud[r][k] = U[r][k] * d[k];
    // (M00, M01), (M11, M12), (M02, M22)
    float2 m0 = make_float2(0.0f, 0.0f), m1 = m0, m2 = m0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        m0 = __ffma2_rn(make_float2(Ud[0][k], Ud[0][k]), make_float2(U[0][k], U[1][k]), m0);
        m1 = __ffma2_rn(make_float2(Ud[1][k], Ud[1][k]), make_float2(U[1][k], U[2][k]), m1);
        m2 = __ffma2_rn(make_float2(Ud[0][k], Ud[2][k]), make_float2(U[2][k], U[2][k]), m2);
    }
    M[0][0] = m0.x;
    M[0][1] = M[1][0] = m0.y;
    M[1][1] = m1.x;
    M[1][2] = M[2][1] = m1.y;
    M[0][2] = M[2][0] = m2.x;
    M[2][2] = m2.y;
}

// P = A B for 3x3 matrices, columns 0 and 1 as packed FP32x2 pairs
__device__ __forceinline__ void matmul3(const float (&A)[3][3], const float (&B)[3][3], float (&P)[3][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float2 p01 = __fmul2_rn(make_float2(A[a][0], A[a][0]), make_float2(B[0][0], B[0][1]));
        p01 = __ffma2_rn(make_float2(A[a][1], A[a][1]), make_float2(B[1][0], B[1][1]), p01);
        p01 = __ffma2_rn(make_float2(A[a][2], A[a][2]), make_float2(B[2][0], B[2][1]), p01);
        P[a][0] = p01.x;
        P[a][1] = p01.y;
        P[a][2] = fmaf(A[a][2], B[2][2], fmaf(A[a][1], B[1][2], A[a][0] * B[0][2]));
    }
}

// ------------------------------------------------------------------------ constitutive update
//
// Plasticine: fixed-corotated elasticity, tau = 2 mu (F - R) F^T + lambda J (J - 1) I, with a von Mises
// return map in Hencky strain: eps = log sig, the deviatoric part of eps is pulled back onto the sphere
// of radius tau_Y / (2 mu) when it lies outside, the trace is kept, F = U exp(eps) V^T. With the polar
// data of the trial F at hand, the stress of the returned F is U diag(d) U^T with
// d_i = 2 mu (s_i - 1) s_i + lambda J (J - 1), s = returned singular values, J = s0 s1 s2.

struct Material {
    float mu, lambda, yield_radius;  // yield_radius = tau_Y / (2 mu)
    float p_mass, stress_scale;      // stress_scale = -dt V0 4 / dx^2
};

// In: trial F (overwritten by the returned F). Out: Kirchhoff stress tau. Returns flag bits.
__device__ __forceinline__ uint32_t plastic_update_and_stress(float (&F)[3][3], const Material& m,
                                                              float (&tau)[3][3]) {
    float U[3][3], sig[3];
    polar_data(F, U, sig);
    uint32_t flags = 0;
    float eps[3];
    bool clamp = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float s = sig[i];
        if (s < 1e-6f) { s = 1e-6f; clamp = true; }
        eps[i] = __logf(s);
    }
    const float tr3 = (eps[0] + eps[1] + eps[2]) * (1.0f / 3.0f);
    const float dev[3] = {eps[0] - tr3, eps[1] - tr3, eps[2] - tr3};
    const float dn2 = dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2];
    const float rdn = rsqrtf(fmaxf(dn2, 1e-30f));
    const float dgamma = dn2 * rdn - m.yield_radius;
    float s[3] = {sig[0], sig[1], sig[2]};
    if (dgamma > 0.0f || clamp) {
        if (dgamma > 0.0f) {
            const float k = dgamma * rdn;
#pragma unroll
            for (int i = 0; i < 3; ++i) eps[i] -= k * dev[i];
        }
        // F <- U diag(s' / sig) U^T F
        float r[3], M[3][3], Fn[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            s[i] = __expf(eps[i]);
            const float g = fabsf(sig[i]) > 1e-30f ? sig[i] : 1e-30f;
            r[i] = __fdividef(s[i], g);
        }
        sym_from_eig(U, r, M);
        matmul3(M, F, Fn);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int c = 0; c < 3; ++c) F[a][c] = Fn[a][c];
        if (clamp) flags |= 0x4u;
    }
    const float J = s[0] * s[1] * s[2];
    const float vol = m.lambda * J * (J - 1.0f);
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = 2.0f * m.mu * (s[i] - 1.0f) * s[i] + vol;
    sym_from_eig(U, d, tau);
    return flags;
}

// Stress of a given (already returned) F, used by the standalone particle-to-grid passes.
__device__ __forceinline__ void fixed_corotated_stress(const float (&F)[3][3], const Material& m, float (&tau)[3][3]) {
    float U[3][3], sig[3];
    polar_data(F, U, sig);
    const float J = sig[0] * sig[1] * sig[2];
    const float vol = m.lambda * J * (J - 1.0f);
    float d[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = 2.0f * m.mu * (sig[i] - 1.0f) * sig[i] + vol;
    sym_from_eig(U, d, tau);
}

// ------------------------------------------------------------------------ colliders
//
// Algorithm 1 copies body poses and velocities once per rigid step; between copies each body moves
// rigidly with those velocities: com(t) = com0 + t v, orientation Rot(w t) R0 (Rodrigues), frame
// origin carried about the centre of mass.

struct SdfVolume {  // a mesh's signed distances on a lattice in the shape frame (type 2)
    const float* data;  // sample (i,j,k) at origin + h (i,j,k), index i + res[0] (j + res[1] k)
    int res[3];
    float origin[3];
    float inv_h;
};

struct ColliderSet {  // as set by the host (one entry per body)
    int type;
    float half[3];
    float friction;
    float pos[3];
    float quat[4];  // w x y z
    float lin[3];
    float ang[3];
    float com[3];
    float reach2;  // squared radius about the frame origin of a ball holding the whole body (padded)
    SdfVolume vol;
};

struct ColliderNow {  // pose at the current substep
    float R[9];       // row-major, local -> world
    float p[3];
    float com[3];
    float lin[3];
    float ang[3];
    float half[3];
    float friction;
    int type;
    float reach2;
    SdfVolume vol;
};

__device__ __forceinline__ void collider_at(const ColliderSet& c, float t, ColliderNow& o) {
    float w = c.quat[0], x = c.quat[1], y = c.quat[2], z = c.quat[3];
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    float R0[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                   2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                   2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    float th[3] = {c.ang[0] * t, c.ang[1] * t, c.ang[2] * t};
    float a = sqrtf(th[0] * th[0] + th[1] * th[1] + th[2] * th[2]);
    float Q[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (a > 0.0f) {
        float k[3] = {th[0] / a, th[1] / a, th[2] / a};
        float K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
        float sa = sinf(a);
        float h = sinf(0.5f * a);
        float ca = 2.0f * h * h;  // 1 - cos a
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float k2 = K[i * 3 + 0] * K[0 * 3 + j] + K[i * 3 + 1] * K[1 * 3 + j] + K[i * 3 + 2] * K[2 * 3 + j];
                Q[i * 3 + j] += sa * K[i * 3 + j] + ca * k2;
            }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            o.R[i * 3 + j] = Q[i * 3 + 0] * R0[0 * 3 + j] + Q[i * 3 + 1] * R0[1 * 3 + j] + Q[i * 3 + 2] * R0[2 * 3 + j];
    float d[3] = {c.pos[0] - c.com[0], c.pos[1] - c.com[1], c.pos[2] - c.com[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        o.com[i] = c.com[i] + t * c.lin[i];
        o.p[i] = o.com[i] + Q[i * 3] * d[0] + Q[i * 3 + 1] * d[1] + Q[i * 3 + 2] * d[2];
        o.lin[i] = c.lin[i];
        o.ang[i] = c.ang[i];
        o.half[i] = c.half[i];
    }
    o.friction = c.friction;
    o.type = c.type;
    o.reach2 = c.reach2;
    o.vol = c.vol;
}

// Trilinear interpolation of an SDF volume at the shape-frame point l (Sec. 3 keeps one per mesh as a
// 3-D texture; here plain loads and FP32 weights, since texture filtering quantises the weights):
// the value, and the interpolant's gradient along each axis as the blend of the cell's four edge
// differences. Returns false outside the lattice.
__device__ __forceinline__ bool sdf_volume(const SdfVolume& V, const float l[3], float& phi, float g[3]) {
    int c[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float u = (l[a] - V.origin[a]) * V.inv_h;
        if (!(u >= 0.0f) || u > (float)(V.res[a] - 1)) return false;
        c[a] = min((int)floorf(u), V.res[a] - 2);
        f[a] = u - (float)c[a];
    }
    const size_t sx = 1, sy = (size_t)V.res[0], sz = (size_t)V.res[0] * V.res[1];
    const float* b = V.data + c[0] + sy * c[1] + sz * c[2];
    float s[2][2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 2; ++k) s[i][j][k] = __ldg(b + i * sx + j * sy + k * sz);
    float val = 0.0f;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 2; ++k)
                val += (i ? f[0] : 1.0f - f[0]) * (j ? f[1] : 1.0f - f[1]) * (k ? f[2] : 1.0f - f[2]) * s[i][j][k];
    g[0] = g[1] = g[2] = 0.0f;
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            g[0] += (e ? f[1] : 1.0f - f[1]) * (o ? f[2] : 1.0f - f[2]) * (s[1][e][o] - s[0][e][o]);
            g[1] += (e ? f[0] : 1.0f - f[0]) * (o ? f[2] : 1.0f - f[2]) * (s[e][1][o] - s[e][0][o]);
            g[2] += (e ? f[0] : 1.0f - f[0]) * (o ? f[1] : 1.0f - f[1]) * (s[e][o][1] - s[e][o][0]);
        }
    phi = val;
#pragma unroll
    for (int a = 0; a < 3; ++a) g[a] *= V.inv_h;
    return true;
}

// Signed distance and world-space outward normal of point xw (analytic box / capsule, SDF volume;
// Sec. 3). A point outside a volume's lattice is outside the body: phi = 1e30, no normal.
__device__ __forceinline__ float collider_sdf(const ColliderNow& c, const float xw[3], float n[3]) {
    float d[3] = {xw[0] - c.p[0], xw[1] - c.p[1], xw[2] - c.p[2]};
    float l[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) l[i] = c.R[i] * d[0] + c.R[3 + i] * d[1] + c.R[6 + i] * d[2];
    float nl[3] = {0.0f, 0.0f, 0.0f};
    float phi;
    if (c.type == 0) {
        float q[3], qo[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            q[i] = fabsf(l[i]) - c.half[i];
            qo[i] = fmaxf(q[i], 0.0f);
        }
        float outside = sqrtf(qo[0] * qo[0] + qo[1] * qo[1] + qo[2] * qo[2]);
        // axis of the largest q (first on ties), chosen with selects so nothing is indexed at run time
        const bool a1 = q[1] > q[0];
        const float q01 = a1 ? q[1] : q[0];
        const bool a2 = q[2] > q01;
        const float qmax = a2 ? q[2] : q01;
        phi = outside + fminf(qmax, 0.0f);
        if (outside > 0.0f) {
            float r = 1.0f / outside;
#pragma unroll
            for (int i = 0; i < 3; ++i) nl[i] = (l[i] >= 0.0f ? 1.0f : -1.0f) * qo[i] * r;
        } else {
            const bool on[3] = {!a1 && !a2, a1 && !a2, a2};
#pragma unroll
            for (int i = 0; i < 3; ++i) nl[i] = on[i] ? (l[i] >= 0.0f ? 1.0f : -1.0f) : 0.0f;
        }
    } else if (c.type == 2) {
        float g[3];
        if (!sdf_volume(c.vol, l, phi, g)) {
            phi = 1e30f;
        } else {
            const float gl = sqrtf(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            if (gl > 0.0f) {
                const float r = 1.0f / gl;
                nl[0] = g[0] * r; nl[1] = g[1] * r; nl[2] = g[2] * r;
            }
        }
    } else {
        float r = c.half[0], h = c.half[1];
        float cz = fminf(fmaxf(l[2], -h), h);
        float e[3] = {l[0], l[1], l[2] - cz};
        float el = sqrtf(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        phi = el - r;
        if (el > 0.0f) {
            float ri = 1.0f / el;
            nl[0] = e[0] * ri; nl[1] = e[1] * ri; nl[2] = e[2] * ri;
        } else {
            nl[0] = 1.0f;
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) n[i] = c.R[i * 3] * nl[0] + c.R[i * 3 + 1] * nl[1] + c.R[i * 3 + 2] * nl[2];
    return phi;
}

// Sums kept as unevaluated FP32 pairs: hi + lo carries about 48 significant bits. An addition is
// Knuth's TwoSum of the high parts (s + e equals a.hi + b.hi exactly), the low parts added to that
// error, then Dekker's Fast2Sum to renormalise. The device-wide mass and momentum sums reduce these
// instead of FP64 values: this part's FP64 pipe is a small fraction of its FP32 one, and a dependent
// tree of FP64 adds and shuffles stalls on it.
struct Pair {
    float hi, lo;
};

__device__ __forceinline__ Pair pair_add(Pair a, Pair b) {
    const float s = a.hi + b.hi;
    const float bv = s - a.hi;
    const float e = ((a.hi - (s - bv)) + (b.hi - bv)) + (a.lo + b.lo);
    const float hi = s + e;
    return Pair{hi, e - (hi - s)};
}

__device__ __forceinline__ Pair pair_add(Pair a, float b) { return pair_add(a, Pair{b, 0.0f}); }

__device__ __forceinline__ Pair pair_shfl_xor(Pair a, int off) {
    return Pair{__shfl_xor_sync(0xffffffffu, a.hi, off), __shfl_xor_sync(0xffffffffu, a.lo, off)};
}

__device__ __forceinline__ double pair_value(Pair a) { return (double)a.hi + (double)a.lo; }

}  // namespace mpm
