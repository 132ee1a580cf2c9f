// lbm_kernels.cuh -- CUDA kernels of the fractional-step MRT lattice Boltzmann
// update (Zhang, Guo & Li, arXiv:1812.02459), written for sm_103a.
//
// The update is a chain of stencils, so every pass below is a tile kernel:
// a CTA stages the tile of its inputs plus the halo its stencils need in
// shared memory (periodic wrap or halfway-wall mirror), computes, and writes
// its tile once.  Arithmetic type T is double or float; populations are
// stored in S (T itself, or bf16 / fp16 in the reduced-storage modes).
//
// Lattice directions (Sec. III.A Eq. D2Q9):
//   c0=(0,0) c1=(1,0) c2=(0,1) c3=(-1,0) c4=(0,-1) c5=(1,1) c6=(-1,1) c7=(-1,-1) c8=(1,-1)
// Moment basis: the rows of Eq. (D2Q9MRT), m = (rho, e, eps, jx, qx, jy, qy, pxx, pxy).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// ---------------------------------------------------------------------------
// Population storage codecs.
// ---------------------------------------------------------------------------
template <typename S, typename T> struct Codec {
    static __device__ __forceinline__ T load(S v) { return (T)v; }
    static __device__ __forceinline__ S store(T v) { return (S)v; }
};
template <> struct Codec<__nv_bfloat16, float> {
    static __device__ __forceinline__ float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ __nv_bfloat16 store(float v) { return __float2bfloat16_rn(v); }
};
// fp16 words hold the value times 2^14: the stored deviations span about
// 1e-8 .. 3e-2, which the scaling moves into fp16's normal range
// [6.1e-5, 65504] (bf16 shares float's exponent range and needs no scaling).
template <> struct Codec<__half, float> {
    static __device__ __forceinline__ float load(__half v) { return __half2float(v) * (1.0f / 16384.0f); }
    static __device__ __forceinline__ __half store(float v) { return __float2half_rn(v * 16384.0f); }
};

// ---------------------------------------------------------------------------
// Model constants handed to every kernel (by value).
// ---------------------------------------------------------------------------
template <typename T> struct KP {
    int nx, ny, px, py;
    long long N;
    unsigned N32;            // N as 32-bit (9 N < 2^32 is enforced on the host)
    T kappa, beta;           // free-energy coefficients (Sec. II.A)
    T eta, M, lambda, W;     // CH equilibrium parameter, mobility, profile weight, width
    int flux_corr;
    T rhoH, rhoL, muH, muL;  // densities and dynamic viscosities of the two fluids
    T drho;                  // (rho_H - rho_L)/2 = d rho / d phi
    T sf[9], sg[9];          // relaxation rates (sg[7], sg[8] set per node)
    T gx, gy;
    T g_rho_ref;             // gravity acts on rho - g_rho_ref
    T eps2;                  // regularisation of |grad phi|^2
    T two_over_W;            // 2/W
    T fd[6];                 // filter coefficients d_0..d_5
    T fa;                    // filter intensity
    int fR;                  // filter half-width (0 = off)
};

// Map a coordinate onto [0,n): periodic wrap, or reflection about the
// halfway walls (-1/2 and n-1/2), which repeats with period 2n; `flip`
// reports an odd number of reflections (sign change of an odd field).
__device__ __forceinline__ int map_axis(int k, int n, int periodic, int &flip)
{
    if ((unsigned)k < (unsigned)n) { flip = 0; return k; }   // inside: the common case
    if (periodic) {
        int r = k % n;
        if (r < 0) r += n;
        flip = 0;
        return r;
    }
    int p = 2 * n;
    int m = k % p;
    if (m < 0) m += p;
    if (m < n) { flip = 0; return m; }
    flip = 1;
    return p - 1 - m;
}

// Asynchronous global -> shared copy of one element (cp.async); the copies
// of a tile are all in flight together and complete at tiles_ready().
template <int B> __device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (B == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// Wait for this thread's asynchronous copies, then for the whole CTA.
__device__ __forceinline__ void tiles_ready()
{
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
}

// Stage a window whose coordinates may leave the domain: each element is
// mapped through the periodic wrap or the wall mirror (synchronous copies).
template <typename T, int WS, int HS>
__device__ __forceinline__ void load_tile_mapped(T *s, const T *__restrict__ g, int x0, int y0, const KP<T> &P,
                                                 bool odd)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < HS; r += nw) {
        int fy;
        const int gy = map_axis(y0 + r, P.ny, P.py, fy);
        const T *row = g + (long long)gy * P.nx;
#pragma unroll
        for (int c = lane; c < WS; c += 32) {
            int fx;
            const int gx = map_axis(x0 + c, P.nx, P.px, fx);
            const T v = __ldg(row + gx);
            s[r * WS + c] = (odd && (fx ^ fy)) ? -v : v;
        }
    }
}

// Stage a (WS x HS) window of a scalar field whose top-left corner is global
// (x0, y0) into shared memory s[HS][WS]; odd fields change sign in mirrors.
// Each warp copies whole rows (lanes along x), so no per-element division
// and at most one coordinate mapping per element on boundary tiles.  Windows
// inside the domain are copied asynchronously: call tiles_ready() before use.
template <typename T, int WS, int HS>
__device__ __forceinline__ void load_tile(T *s, const T *__restrict__ g, int x0, int y0,
                                          const KP<T> &P, bool odd)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (x0 >= 0 && y0 >= 0 && x0 + WS <= P.nx && y0 + HS <= P.ny) {
        const T *row = g + ((long long)y0 * P.nx + x0) + warp * P.nx;
        T *srow = s + warp * WS;
        const int rstep = nw * P.nx;
        for (int r = warp; r < HS; r += nw, row += rstep, srow += nw * WS) {
#pragma unroll
            for (int c = lane; c < WS; c += 32) cp_async<sizeof(T)>(&srow[c], row + c);
        }
        return;
    }
    load_tile_mapped<T, WS, HS>(s, g, x0, y0, P, odd);
}

// Isotropic first derivatives and Laplacian on a D2Q9 neighbourhood
// (Sec. III.B Eq. dicretized): with E,W,N,S the axis neighbours and
// NE,NW,SW,SE the diagonals,
//   d_x = (E-W)/3 + (NE-NW-SW+SE)/12,  d_y = (N-S)/3 + (NE+NW-SW-SE)/12,
//   lap = 2/3 (E+W+N+S) + 1/6 (NE+NW+SW+SE) - 10/3 C.
template <typename T, int WS>
__device__ __forceinline__ void iso_grad(const T *s, int i, T &dx, T &dy)
{
    const T E = s[i + 1], Wv = s[i - 1], N = s[i + WS], S = s[i - WS];
    const T NE = s[i + WS + 1], NW = s[i + WS - 1], SW = s[i - WS - 1], SE = s[i - WS + 1];
    dx = (E - Wv) * T(1.0 / 3.0) + (NE - NW - SW + SE) * T(1.0 / 12.0);
    dy = (N - S) * T(1.0 / 3.0) + (NE + NW - SW - SE) * T(1.0 / 12.0);
}
template <typename T, int WS>
__device__ __forceinline__ T iso_lap(const T *s, int i)
{
    const T ax = s[i + 1] + s[i - 1] + s[i + WS] + s[i - WS];
    const T dg = s[i + WS + 1] + s[i + WS - 1] + s[i - WS - 1] + s[i - WS + 1];
    return ax * T(2.0 / 3.0) + dg * T(1.0 / 6.0) - s[i] * T(10.0 / 3.0);
}

// Fourth-order central differences (Sec. III.A Eq. fourOrder_FDM) and the
// five-point fourth-order second derivative.
template <typename T, int STRIDE>
__device__ __forceinline__ T fd4_d1(const T *s, int i)
{
    return (s[i - 2 * STRIDE] - T(8) * s[i - STRIDE] + T(8) * s[i + STRIDE] - s[i + 2 * STRIDE]) *
           T(1.0 / 12.0);
}
template <typename T, int STRIDE>
__device__ __forceinline__ T fd4_d2(const T *s, int i)
{
    return (-s[i - 2 * STRIDE] + T(16) * s[i - STRIDE] - T(30) * s[i] + T(16) * s[i + STRIDE] -
            s[i + 2 * STRIDE]) *
           T(1.0 / 12.0);
}

// Reciprocal and reciprocal square root: IEEE in FP64 (the parity build).
// In FP32 the reciprocal is the hardware approximation refined by one
// Newton step, r + r (1 - x r), which leaves it within about half an ulp
// at two FMAs (the correctly rounded __frcp_rn measured 13% slower in the
// collide kernel); the reciprocal square root (the normal n of the FD
// correction) is the hardware approximation (<= 2 ulp).
__device__ __forceinline__ float rcp(float x)
{
    const float r = __fdividef(1.0f, x);
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return 1.0 / sqrt(x); }

// The rounding error of s = a + b (Knuth's TwoSum, exact in IEEE arithmetic):
// a + b = s + err.  phi is carried as phi_hi + phi_lo, each step adding its
// increment r to phi_hi and keeping what the rounding of the sum drops.
template <typename T> __device__ __forceinline__ T two_sum_err(T a, T b, T s)
{
    const T bp = s - a, ap = s - bp;
    return (a - ap) + (b - bp);
}

// Density, its reciprocal and the kinematic viscosity at a node (Sec. II.B
// Eq. rho, Sec. III.B Eq. dynamic_vis), with phi clamped to [-1,1] here only.
template <typename T>
__device__ __forceinline__ void rho_nu(const KP<T> &P, T phi, T &rho, T &irho, T &nu)
{
    T c = phi < T(-1) ? T(-1) : (phi > T(1) ? T(1) : phi);
    T hp = (T(1) + c) * T(0.5), hm = (T(1) - c) * T(0.5);
    rho = P.rhoH * hp + P.rhoL * hm;
    irho = rcp(rho);
    nu = (P.muH * hp + P.muL * hm) * irho;
}

// Lattice weights (Sec. III.A, below Eq. D2Q9).
__device__ __forceinline__ float lattice_w(int q) { return q == 0 ? 4.0f / 9.0f : (q < 5 ? 1.0f / 9.0f : 1.0f / 36.0f); }
template <typename T> __device__ __forceinline__ T lattice_w_t(int q)
{
    return q == 0 ? T(4) / T(9) : (q < 5 ? T(1) / T(9) : T(1) / T(36));
}

// Reduced-precision population storage (S narrower than T).  Only the
// deviations from the rest equilibria are stored in S: the CH rest
// equilibrium is (phi, 0, ..., 0), so f_1..f_8 are stored as they are; the NS
// rest equilibrium is 3 w_i p, so g_i - 3 w_i p_hat is stored for i = 1..8.
// The rest populations are rebuilt from the post-stream moments kept in T,
// f_0 = phi_bar - sum_{i>0} f_i and g_0 = 3 p_hat - sum_{i>0} g_i, so sum f and
// sum g are carried in T whatever the rounding of the stored words.
template <typename T, typename S> struct Mixed {
    static constexpr bool on = sizeof(S) < sizeof(T);
};

// The velocity part of the NS equilibrium g_q = w_q (3 p + s_q(u)) of
// Eq. (geq), without its weight: s_q(u) = 3 c.u + 9/2 (c.u)^2 - 3/2 u.u.
// Reduced-precision storage keeps g_q - w_q (3 p_hat + s_q(u^n)), the NS
// populations less their equilibrium at the node's post-stream p_hat and the
// velocity u^n they were collided with, so that the 16-bit words carry only
// the non-equilibrium part; a reader adds the equilibrium back from p_hat and
// u^n (the u^{n-1} slot of the next step).
template <typename T> __host__ __device__ __forceinline__ T s_eq(int q, T u0, T u1)
{
    const int cx = (q == 1 || q == 5 || q == 8) ? 1 : ((q == 3 || q == 6 || q == 7) ? -1 : 0);
    const int cy = (q == 2 || q == 5 || q == 6) ? 1 : ((q == 4 || q == 7 || q == 8) ? -1 : 0);
    const T cu = T(cx) * u0 + T(cy) * u1;
    return cu * (T(3) + T(4.5) * cu) - T(1.5) * (u0 * u0 + u1 * u1);
}

// Moment transform m = M f with the rows of Eq. (D2Q9MRT).
template <typename T>
__device__ __forceinline__ void to_moments(const T f[9], T m[9])
{
    const T a = f[1] + f[2] + f[3] + f[4], d = f[5] + f[6] + f[7] + f[8];
    m[0] = f[0] + a + d;
    m[1] = T(-4) * f[0] - a + T(2) * d;
    m[2] = T(4) * f[0] - T(2) * a + d;
    const T d58 = f[5] - f[6] - f[7] + f[8];
    m[3] = f[1] - f[3] + d58;
    m[4] = T(2) * (f[3] - f[1]) + d58;
    const T d56 = f[5] + f[6] - f[7] - f[8];
    m[5] = f[2] - f[4] + d56;
    m[6] = T(2) * (f[4] - f[2]) + d56;
    m[7] = f[1] - f[2] + f[3] - f[4];
    m[8] = f[5] - f[6] + f[7] - f[8];
}

// Inverse transform f = M^{-1} m; the rows of M are orthogonal with squared
// norms (9,36,36,6,12,6,12,4,4), so M^{-1} = M^T diag(1/norm^2).
template <typename T>
__device__ __forceinline__ void from_moments(const T m[9], T f[9])
{
    const T r = m[0] * T(1.0 / 9.0), e = m[1] * T(1.0 / 36.0), ep = m[2] * T(1.0 / 36.0);
    const T jx = m[3] * T(1.0 / 6.0), qx = m[4] * T(1.0 / 12.0);
    const T jy = m[5] * T(1.0 / 6.0), qy = m[6] * T(1.0 / 12.0);
    const T pxx = m[7] * T(0.25), pxy = m[8] * T(0.25);
    f[0] = r - T(4) * e + T(4) * ep;
    const T ax = r - e - T(2) * ep;
    const T sx = jx - T(2) * qx, sy = jy - T(2) * qy;
    f[1] = ax + sx + pxx;
    f[2] = ax + sy - pxx;
    f[3] = ax - sx + pxx;
    f[4] = ax - sy - pxx;
    const T dg = r + T(2) * e + ep;
    const T tx = jx + qx, ty = jy + qy;
    f[5] = dg + tx + ty + pxy;
    f[6] = dg - tx + ty - pxy;
    f[7] = dg - tx - ty + pxy;
    f[8] = dg + tx - ty - pxy;
}

// ---------------------------------------------------------------------------
// Pass 1: fields and forces at t^n, collision of both lattices, pull
// streaming and the post-stream moments, fused per tile.
//
// For every node of the tile plus a one-node ring the CTA evaluates
//   mu   = 4 beta (phi^3 - phi) - kappa lap phi          (Sec. II.A Eq. chemical)
//   F    = -p grad rho + kappa div(|grad phi|^2 I - grad phi grad phi)
//          + nu (grad u + grad u^T).grad rho + J.grad u + rho g,
//   J    = (d rho/d phi) M grad mu                       (Sec. II.B Eqs. surfaceforce, reformNS)
//   a    = (u^n - u^{n-1}) + u.grad u                    (source of Eq. Fi)
// and collides in moment space:
//   f:  m* = m - S^f (m - m_eq(phi, mu, u)) + (I - S^f/2) M F_i         (Eqs. distribution_CH, feq_CH, Fi)
//   g:  m* = m_eq(p_f, u_f) + (I - S^g)(m - m_eq(p_hat, u_hat)) + (I - S^g/2) M G_i
//        with M G_i = (0, 6 b.u, -6 b.u, Fx/rho, -Fx/rho, Fy/rho, -Fy/rho,
//                      2(bx ux - by uy), by ux + bx uy),  b = F/rho - grad p   (Eq. Gi, App. A)
// The post-collision populations of tile+ring sit in shared memory, so each
// tile node pulls f_i(x) = f*_i(x - c_i) (halfway bounce-back at walls),
// writes it once, and emits phi_bar = sum f (Eq. compute_phi),
// p_hat = cs^2 sum g (Eq. p) and j = sum c g (first part of Eq. u).
// phi_bar is emitted as its increment dbar = phi_bar - phi over the phi the
// collision used: the CH populations are collided as deviations from
// phi e_0 (the moments of phi e_0 removed from m and m_eq), so dbar is a sum
// of small terms and keeps its relative precision in FP32, where an O(1)
// phi_bar would lose a unit roundoff of phi to every step.
// ---------------------------------------------------------------------------
template <int TX, int TY> struct CSGeom {
    static constexpr int W3 = TX + 6, H3 = TY + 6;   // phi window (ring 3)
    static constexpr int W2 = TX + 4, H2 = TY + 4;   // p, u windows; mu, grad phi (ring 2)
    static constexpr int W1 = TX + 2, H1 = TY + 2;   // collision region (ring 1)
    static constexpr int A3 = W3 * H3, A2 = W2 * H2, A1 = W1 * H1;
    static constexpr int NSCALAR = A3 + 9 * A2 + 18 * A1;
};

// Surface force kappa div(T) from the tensor components stored in a window
// of row stride WS: txx = gy^2, txy = -gx gy, tyy = gx^2 (isotropic divergence).
template <typename T, int WS>
__device__ __forceinline__ void surface_force_t(const T *txx, const T *txy, const T *tyy, int i, T kappa,
                                                T &Fx, T &Fy)
{
    T dxx, dxy_x, dxy_y, dyy;
    iso_grad<T, WS>(txy, i, dxy_x, dxy_y);
    dxx = (txx[i + 1] - txx[i - 1]) * T(1.0 / 3.0) +
          (txx[i + WS + 1] - txx[i + WS - 1] - txx[i - WS - 1] + txx[i - WS + 1]) * T(1.0 / 12.0);
    dyy = (tyy[i + WS] - tyy[i - WS]) * T(1.0 / 3.0) +
          (tyy[i + WS + 1] + tyy[i + WS - 1] - tyy[i - WS - 1] - tyy[i - WS + 1]) * T(1.0 / 12.0);
    Fx = kappa * (dxx + dxy_y);
    Fy = kappa * (dxy_x + dyy);
}

// Surface force kappa div(T), T = |grad phi|^2 I - grad phi grad phi
// = (gy^2, -gx gy; -gx gy, gx^2), isotropic divergence from grad phi stored
// at the eight neighbours of index i of a window of row stride WS.
template <typename T, int WS>
__device__ __forceinline__ void surface_force(const T *sgx, const T *sgy, int i, T kappa, T &Fx, T &Fy)
{
    const int nb[8] = {i + 1, i - 1, i + WS, i - WS, i + WS + 1, i + WS - 1, i - WS - 1, i - WS + 1};
    T txx[8], txy[8], tyy[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const T a = sgx[nb[k]], b = sgy[nb[k]];
        txx[k] = b * b;
        txy[k] = -a * b;
        tyy[k] = a * a;
    }
    // neighbour order: E, W, N, S, NE, NW, SW, SE
    const T dxx = (txx[0] - txx[1]) * T(1.0 / 3.0) + (txx[4] - txx[5] - txx[6] + txx[7]) * T(1.0 / 12.0);
    const T dyxy = (txy[2] - txy[3]) * T(1.0 / 3.0) + (txy[4] + txy[5] - txy[6] - txy[7]) * T(1.0 / 12.0);
    const T dxxy = (txy[0] - txy[1]) * T(1.0 / 3.0) + (txy[4] - txy[5] - txy[6] + txy[7]) * T(1.0 / 12.0);
    const T dyyy = (tyy[2] - tyy[3]) * T(1.0 / 3.0) + (tyy[4] + tyy[5] - tyy[6] - tyy[7]) * T(1.0 / 12.0);
    Fx = kappa * (dxx + dyxy);
    Fy = kappa * (dxxy + dyyy);
}

// FAST: the relaxation rates hold their defaults -- s_f = 1 except s_f[3],
// s_f[5] (= 1/tau_f), s_g[0..3] = s_g[5] = 1 -- so every moment relaxed at
// rate 1 is set straight to m_eq + m_source/2 and only the moments relaxed at
// other rates are formed from the incoming populations.
template <typename T, typename S, int TX, int TY, bool FAST>
__global__ void __launch_bounds__((TX + 2) * (TY + 2), sizeof(T) == 4 ? 3 : 2)
k_collide_stream(KP<T> P, const S *__restrict__ fin, const S *__restrict__ gin,
                 S *__restrict__ fout, S *__restrict__ gout,
                 const T *__restrict__ phi, const T *__restrict__ pfl,
                 const T *__restrict__ ux, const T *__restrict__ uy,
                 const T *__restrict__ upx, const T *__restrict__ upy,
                 const T *__restrict__ uhx, const T *__restrict__ uhy,
                 const T *__restrict__ phi_prev, const T *__restrict__ dbar_old,
                 const T *__restrict__ phat_old, const T *__restrict__ philo,
                 T *__restrict__ dbar, T *__restrict__ phat,
                 T *__restrict__ jxo, T *__restrict__ jyo)
{
    // One thread per node of the collision region (tile + ring 1): the
    // launch uses exactly A1 threads.  The CH populations are carried as
    // deviations from the rest state of the node's phi: f'_0 = f_0 - phi,
    // f'_i = f_i (i > 0), so their post-stream sum is the small increment
    // dbar = phi_bar - phi, free of the rounding of an O(1) sum.  phi_prev,
    // dbar_old and phat_old give the post-stream moments of the stored
    // populations (phi_bar = phi_prev + dbar_old, p_hat); they are read only
    // when the populations are stored in reduced precision.  philo (FP32
    // handles, else NULL) holds the low part of phi = phi_hi + phi_lo: the
    // collision relaxes m_0 to the whole of it, so phi_lo enters dbar.
    using G = CSGeom<TX, TY>;
    constexpr int W3 = G::W3, W2 = G::W2, H2 = G::H2, W1 = G::W1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_phi = reinterpret_cast<T *>(smem_raw);
    T *s_p = s_phi + G::A3;
    T *s_ux = s_p + G::A2;
    T *s_uy = s_ux + G::A2;
    T *s_mu = s_uy + G::A2;
    T *s_gx = s_mu + G::A2;
    T *s_gy = s_gx + G::A2;
    T *s_txx = s_gy + G::A2;
    T *s_txy = s_txx + G::A2;
    T *s_tyy = s_txy + G::A2;
    T *s_f = s_tyy + G::A2;      // [9][A1]
    T *s_g = s_f + 9 * G::A1;    // [9][A1]

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const long long N = P.N;

    // this thread's collision node, and its populations requested up front so
    // that their latency overlaps the staging and the first stencil phase
    const int t = threadIdx.x;
    const int ly = t / W1, lx = t - ly * W1;
    const int X = x0 - 1 + lx, Y = y0 - 1 + ly;
    const bool ghost = (!P.px && (X < 0 || X >= P.nx)) || (!P.py && (Y < 0 || Y >= P.ny));
    int fxm, fym;
    const int gidx = map_axis(Y, P.ny, P.py, fym) * P.nx + map_axis(X, P.nx, P.px, fxm);
    T f[9], g[9], upx_ = T(0), upy_ = T(0), uhx_ = T(0), uhy_ = T(0), pprev = T(0), plo = T(0);
    if (!ghost) {
        const unsigned N32 = P.N32;
        upx_ = __ldg(&upx[gidx]);
        upy_ = __ldg(&upy[gidx]);
        if constexpr (Mixed<T, S>::on) {
            T sf = T(0), sg = T(0);
            const T ph0 = __ldg(&phat_old[gidx]);
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                const unsigned o = (unsigned)gidx + (unsigned)q * N32;
                f[q] = Codec<S, T>::load(__ldg(&fin[o]));
                g[q] = Codec<S, T>::load(__ldg(&gin[o])) + T(lattice_w(q)) * (T(3) * ph0 + s_eq(q, upx_, upy_));
                sf += f[q];
                sg += g[q];
            }
            // f_0 - phi_prev; the node's phi is subtracted once the window is staged
            f[0] = __ldg(&dbar_old[gidx]) - sf;
            pprev = __ldg(&phi_prev[gidx]);
            g[0] = T(3) * ph0 - sg;
        } else {
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const unsigned o = (unsigned)gidx + (unsigned)q * N32;
                f[q] = Codec<S, T>::load(__ldg(&fin[o]));
                g[q] = Codec<S, T>::load(__ldg(&gin[o]));
            }
        }
        if (philo) plo = __ldg(&philo[gidx]);
        uhx_ = __ldg(&uhx[gidx]);
        uhy_ = __ldg(&uhy[gidx]);
    }

    load_tile<T, G::W3, G::H3>(s_phi, phi, x0 - 3, y0 - 3, P, false);
    load_tile<T, W2, H2>(s_p, pfl, x0 - 2, y0 - 2, P, false);
    load_tile<T, W2, H2>(s_ux, ux, x0 - 2, y0 - 2, P, true);
    load_tile<T, W2, H2>(s_uy, uy, x0 - 2, y0 - 2, P, true);
    tiles_ready();

    // chemical potential and grad phi on tile + ring 2
    for (int k = threadIdx.x; k < G::A2; k += blockDim.x) {
        int ky = k / W2, kx = k - ky * W2;
        int i3 = (ky + 1) * W3 + (kx + 1);
        T ph = s_phi[i3];
        s_mu[k] = T(4) * P.beta * (ph * ph * ph - ph) - P.kappa * iso_lap<T, W3>(s_phi, i3);
        T gx, gy;
        iso_grad<T, W3>(s_phi, i3, gx, gy);
        s_gx[k] = gx;
        s_gy[k] = gy;
        s_txx[k] = gy * gy;
        s_txy[k] = -gx * gy;
        s_tyy[k] = gx * gx;
    }
    __syncthreads();

    // forces and collision of this thread's node
    if (!ghost) {   // beyond a wall: never pulled (bounce-back instead)
        const int i2 = (ly + 1) * W2 + (lx + 1);
        const int i3 = (ly + 2) * W3 + (lx + 2);

        const T ph = s_phi[i3];
        f[0] = Mixed<T, S>::on ? (pprev - ph) + f[0] : f[0] - ph;   // f'_0
        T rho, ir, nu;
        rho_nu(P, ph, rho, ir, nu);
        const T mu = s_mu[i2];
        const T grx = P.drho * s_gx[i2], gry = P.drho * s_gy[i2];
        T dmx, dmy;
        iso_grad<T, W2>(s_mu, i2, dmx, dmy);
        const T Jx = P.drho * P.M * dmx, Jy = P.drho * P.M * dmy;
        T Fsx, Fsy;
        surface_force_t<T, W2>(s_txx, s_txy, s_tyy, i2, P.kappa, Fsx, Fsy);
        const T pc = s_p[i2];
        T dpx, dpy, dxux, dyux, dxuy, dyuy;
        iso_grad<T, W2>(s_p, i2, dpx, dpy);
        iso_grad<T, W2>(s_ux, i2, dxux, dyux);
        iso_grad<T, W2>(s_uy, i2, dxuy, dyuy);
        const T u0 = s_ux[i2], u1 = s_uy[i2];
        const T Sxx = T(2) * dxux, Sxy = dyux + dxuy, Syy = T(2) * dyuy;
        const T Fx = -pc * grx + Fsx + nu * (Sxx * grx + Sxy * gry) + (Jx * dxux + Jy * dyux) + (rho - P.g_rho_ref) * P.gx;
        const T Fy = -pc * gry + Fsy + nu * (Sxy * grx + Syy * gry) + (Jx * dxuy + Jy * dyuy) + (rho - P.g_rho_ref) * P.gy;
        // mirrored ring nodes carry the odd sign of u^{n-1} and u_hat too
        const T sgn = (fxm ^ fym) ? T(-1) : T(1);
        const T ax = (u0 - sgn * upx_) + u0 * dxux + u1 * dyux;
        const T ay = (u1 - sgn * upy_) + u0 * dxuy + u1 * dyuy;
        const T u2 = u0 * u0 + u1 * u1;

        // ---- CH populations, as deviations from phi e_0: the moments of
        // phi e_0, (phi, -4 phi, 4 phi, 0, ...), are left out of m and m_eq
        {
            T m[9];
            const T em = P.eta * mu;
            const T meq[9] = {plo, T(2) * em + T(3) * ph * u2 - T(4) * plo, T(4) * plo - T(3) * em - T(3) * ph * u2,
                              ph * u0, -ph * u0, ph * u1, -ph * u1, ph * (u0 * u0 - u1 * u1), ph * u0 * u1};
            const T mF[9] = {T(0), T(0), T(0), ph * ax, -ph * ax, ph * ay, -ph * ay, T(0), T(0)};
            if constexpr (FAST) {
                const T s = P.sf[3];
                const T m3 = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
                const T m5 = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
#pragma unroll
                for (int k = 0; k < 9; ++k) m[k] = meq[k] + T(0.5) * mF[k];
                m[3] = m3 - s * (m3 - meq[3]) + (T(1) - T(0.5) * s) * mF[3];
                m[5] = m5 - s * (m5 - meq[5]) + (T(1) - T(0.5) * s) * mF[5];
            } else {
                to_moments(f, m);
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    m[k] = m[k] - P.sf[k] * (m[k] - meq[k]) + (T(1) - T(0.5) * P.sf[k]) * mF[k];
            }
            from_moments(m, f);
#pragma unroll
            for (int q = 0; q < 9; ++q) s_f[q * G::A1 + t] = f[q];
        }
        // ---- NS populations
        {
            T m[9];
            const T h0 = sgn * uhx_, h1 = sgn * uhy_;
            const T mef[9] = {T(3) * pc, T(-6) * pc + T(3) * u2, T(3) * pc - T(3) * u2, u0, -u0, u1, -u1,
                              u0 * u0 - u1 * u1, u0 * u1};
            const T bx = Fx * ir - dpx, by = Fy * ir - dpy;
            const T bu = bx * u0 + by * u1;
            const T mG[9] = {T(0), T(6) * bu, T(-6) * bu, Fx * ir, -Fx * ir, Fy * ir, -Fy * ir,
                             T(2) * (bx * u0 - by * u1), by * u0 + bx * u1};
            const T s78 = rcp(nu * T(3) + T(0.5));   // 1/tau_g, tau_g = nu/cs^2 + 1/2
            if constexpr (FAST) {
                // rate-1 moments (0,1,2,3,5) drop the non-equilibrium part,
                // so the unfiltered p_hat is not needed
#pragma unroll
                for (int k = 0; k < 9; ++k) m[k] = mef[k] + T(0.5) * mG[k];
                const T d58 = g[5] - g[6] - g[7] + g[8], d56 = g[5] + g[6] - g[7] - g[8];
                const T m4 = T(2) * (g[3] - g[1]) + d58, m6 = T(2) * (g[4] - g[2]) + d56;
                const T m7 = g[1] - g[2] + g[3] - g[4], m8 = g[5] - g[6] + g[7] - g[8];
                const T s4 = P.sg[4], s6 = P.sg[6];
                m[4] += (T(1) - s4) * (m4 + h0) + (T(0.5) - T(0.5) * s4) * mG[4];
                m[6] += (T(1) - s6) * (m6 + h1) + (T(0.5) - T(0.5) * s6) * mG[6];
                m[7] += (T(1) - s78) * (m7 - (h0 * h0 - h1 * h1)) + (T(0.5) - T(0.5) * s78) * mG[7];
                m[8] += (T(1) - s78) * (m8 - h0 * h1) + (T(0.5) - T(0.5) * s78) * mG[8];
            } else {
                to_moments(g, m);
                const T ph_ = m[0] * T(1.0 / 3.0);          // p_hat = cs^2 sum g
                const T h2 = h0 * h0 + h1 * h1;
                const T meh[9] = {T(3) * ph_, T(-6) * ph_ + T(3) * h2, T(3) * ph_ - T(3) * h2, h0, -h0, h1, -h1,
                                  h0 * h0 - h1 * h1, h0 * h1};
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    const T sk = k < 7 ? P.sg[k] : s78;
                    m[k] = mef[k] + (T(1) - sk) * (m[k] - meh[k]) + (T(1) - T(0.5) * sk) * mG[k];
                }
            }
            from_moments(m, g);
#pragma unroll
            for (int q = 0; q < 9; ++q) s_g[q * G::A1 + t] = g[q];
        }
    }
    __syncthreads();

    // pull streaming for the tile and post-stream moments
    constexpr int cxv[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int cyv[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    for (int k = threadIdx.x; k < TX * TY; k += blockDim.x) {
        const int ky = k / TX, kx = k - ky * TX;
        const int Xn = x0 + kx, Yn = y0 + ky;
        if (Xn >= P.nx || Yn >= P.ny) continue;
        const int nidx = Yn * P.nx + Xn;
        const int c1 = (ky + 1) * W1 + (kx + 1);
        const bool edge = (!P.px && (Xn == 0 || Xn == P.nx - 1)) || (!P.py && (Yn == 0 || Yn == P.ny - 1));
        T fv[9], gv[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            int src = q * G::A1 + c1 - cyv[q] * W1 - cxv[q];
            if (edge) {
                const int SX = Xn - cxv[q], SY = Yn - cyv[q];
                const bool wall = (!P.px && (SX < 0 || SX >= P.nx)) || (!P.py && (SY < 0 || SY >= P.ny));
                if (wall) src = opp[q] * G::A1 + c1;
            }
            fv[q] = s_f[src];
            gv[q] = s_g[src];
        }
        T sf = T(0), sg = T(0), sgx = T(0), sgy = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            sf += fv[q];
            sg += gv[q];
            sgx += T(cxv[q]) * gv[q];
            sgy += T(cyv[q]) * gv[q];
        }
        const T pn = sg * T(1.0 / 3.0);
        const unsigned N32 = P.N32;
        if constexpr (Mixed<T, S>::on) {
            const int iu = (ky + 2) * W2 + (kx + 2);   // u^n of this node in its window
            const T un0 = s_ux[iu], un1 = s_uy[iu];
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                const unsigned o = (unsigned)nidx + (unsigned)q * N32;
                fout[o] = Codec<S, T>::store(fv[q]);
                gout[o] = Codec<S, T>::store(gv[q] - T(lattice_w(q)) * (T(3) * pn + s_eq(q, un0, un1)));
            }
        } else {
            fout[nidx] = Codec<S, T>::store(s_phi[(ky + 3) * W3 + (kx + 3)] + fv[0]);
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                const unsigned o = (unsigned)nidx + (unsigned)q * N32;
                fout[o] = Codec<S, T>::store(fv[q]);
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const unsigned o = (unsigned)nidx + (unsigned)q * N32;
                gout[o] = Codec<S, T>::store(gv[q]);
            }
        }
        dbar[nidx] = sf;
        phat[nidx] = pn;
        jxo[nidx] = sgx;
        jyo[nidx] = sgy;
    }
}

// ---------------------------------------------------------------------------
// Pass 1 of the Cahn-Hilliard part alone, under a prescribed velocity (the
// interface-capturing tests of Sec. IV.A-B, where the flow is given):
// mu = 4 beta (phi^3 - phi) - kappa lap phi, the CH collision with
// f_eq(phi, mu, u) and the source F_i of a = (u - u_prev) + u.grad u
// (Eqs. feq_CH, Fi), pull streaming and dbar = phi_bar - phi.  The NS
// lattice is not touched.  The velocity is u = us * u0 and the previous
// step's up_s * up; one node per thread of the collision region, the general
// relaxation of every moment, populations stored in T.
// ---------------------------------------------------------------------------
template <int TX, int TY> struct CHGeom {
    static constexpr int W2 = TX + 4, H2 = TY + 4;   // phi, u windows (ring 2)
    static constexpr int W1 = TX + 2, H1 = TY + 2;   // collision region (ring 1)
    static constexpr int A2 = W2 * H2, A1 = W1 * H1;
    static constexpr int NSCALAR = 3 * A2 + 9 * A1;
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__((TX + 2) * (TY + 2))
k_collide_ch(KP<T> P, const T *__restrict__ fin, T *__restrict__ fout, const T *__restrict__ phi,
             const T *__restrict__ philo, const T *__restrict__ u0x, const T *__restrict__ u0y, T us,
             const T *__restrict__ upx, const T *__restrict__ upy, T ups, T *__restrict__ dbar)
{
    using G = CHGeom<TX, TY>;
    constexpr int W2 = G::W2, H2 = G::H2, W1 = G::W1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_phi = reinterpret_cast<T *>(smem_raw);
    T *s_ux = s_phi + G::A2;
    T *s_uy = s_ux + G::A2;
    T *s_f = s_uy + G::A2;   // [9][A1]
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int t = threadIdx.x;
    const int ly = t / W1, lx = t - ly * W1;
    const int X = x0 - 1 + lx, Y = y0 - 1 + ly;
    const bool ghost = (!P.px && (X < 0 || X >= P.nx)) || (!P.py && (Y < 0 || Y >= P.ny));
    int fl;
    const int gidx = map_axis(Y, P.ny, P.py, fl) * P.nx + map_axis(X, P.nx, P.px, fl);
    T f[9], plo = T(0), upx_ = T(0), upy_ = T(0);
    if (!ghost) {
#pragma unroll
        for (int q = 0; q < 9; ++q) f[q] = __ldg(&fin[(size_t)gidx + (size_t)q * P.N]);
        if (philo) plo = __ldg(&philo[gidx]);
        upx_ = ups * __ldg(&upx[gidx]);
        upy_ = ups * __ldg(&upy[gidx]);
    }
    load_tile<T, W2, H2>(s_phi, phi, x0 - 2, y0 - 2, P, false);
    load_tile<T, W2, H2>(s_ux, u0x, x0 - 2, y0 - 2, P, true);
    load_tile<T, W2, H2>(s_uy, u0y, x0 - 2, y0 - 2, P, true);
    tiles_ready();

    if (!ghost) {
        const int i2 = (ly + 1) * W2 + (lx + 1);
        const T ph = s_phi[i2];
        const T mu = T(4) * P.beta * (ph * ph * ph - ph) - P.kappa * iso_lap<T, W2>(s_phi, i2);
        T dxux, dyux, dxuy, dyuy;
        iso_grad<T, W2>(s_ux, i2, dxux, dyux);
        iso_grad<T, W2>(s_uy, i2, dxuy, dyuy);
        const T u0 = us * s_ux[i2], u1 = us * s_uy[i2];
        dxux *= us; dyux *= us; dxuy *= us; dyuy *= us;
        const T ax = (u0 - upx_) + u0 * dxux + u1 * dyux;
        const T ay = (u1 - upy_) + u0 * dxuy + u1 * dyuy;
        const T u2 = u0 * u0 + u1 * u1, em = P.eta * mu;
        // deviations from phi_hi e_0, m_0 relaxing to phi_hi + phi_lo (as in k_collide_stream)
        f[0] -= ph;
        const T meq[9] = {plo, T(2) * em + T(3) * ph * u2 - T(4) * plo, T(4) * plo - T(3) * em - T(3) * ph * u2,
                          ph * u0, -ph * u0, ph * u1, -ph * u1, ph * (u0 * u0 - u1 * u1), ph * u0 * u1};
        const T mF[9] = {T(0), T(0), T(0), ph * ax, -ph * ax, ph * ay, -ph * ay, T(0), T(0)};
        T m[9];
        to_moments(f, m);
#pragma unroll
        for (int k = 0; k < 9; ++k) m[k] = m[k] - P.sf[k] * (m[k] - meq[k]) + (T(1) - T(0.5) * P.sf[k]) * mF[k];
        from_moments(m, f);
#pragma unroll
        for (int q = 0; q < 9; ++q) s_f[q * G::A1 + t] = f[q];
    }
    __syncthreads();

    constexpr int cxv[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    constexpr int cyv[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    constexpr int opp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    for (int k = threadIdx.x; k < TX * TY; k += blockDim.x) {
        const int ky = k / TX, kx = k - ky * TX;
        const int Xn = x0 + kx, Yn = y0 + ky;
        if (Xn >= P.nx || Yn >= P.ny) continue;
        const size_t nidx = (size_t)Yn * P.nx + Xn;
        const int c1 = (ky + 1) * W1 + (kx + 1);
        const bool edge = (!P.px && (Xn == 0 || Xn == P.nx - 1)) || (!P.py && (Yn == 0 || Yn == P.ny - 1));
        T sf = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            int src = q * G::A1 + c1 - cyv[q] * W1 - cxv[q];
            if (edge) {
                const int SX = Xn - cxv[q], SY = Yn - cyv[q];
                if ((!P.px && (SX < 0 || SX >= P.nx)) || (!P.py && (SY < 0 || SY >= P.ny))) src = opp[q] * G::A1 + c1;
            }
            const T v = s_f[src];
            sf += v;
            fout[nidx + (size_t)q * P.N] = q == 0 ? s_phi[(ky + 2) * W2 + (kx + 2)] + v : v;
        }
        dbar[nidx] = sf;
    }
}

// ---------------------------------------------------------------------------
// Pass 2: one stage of the TVD-RK3 correction (Sec. III.A Eq. TVD-3order)
//   psi^(k) = a phi_bar + b (psi^(k-1) + L(psi^(k-1))),  L(psi) = div(lambda J_phi + q),
//   J_phi = (|grad psi| - 2(1 - psi^2)/W) n,  q = -M (grad mu_psi . n) n,
//   n = grad psi / |grad psi|,  mu_psi = 4 beta (psi^3 - psi) - kappa lap psi,
// every derivative by fourth-order central differences (Eq. fourOrder_FDM).
// The stages are carried as increments over the step's phi^n: with
// phi_bar = phi^n + dbar and psi^(k) = phi^n + d^(k), a stage computes
//   d^(k) = a dbar + b (d^(k-1) + L(phi^n + d^(k-1)))     (d^(0) = dbar),
// and the last stage writes phi^{n+1} = phi^n + d^(3).  The increments are
// small, so the arithmetic that combines the stages keeps their relative
// precision, and phi is rounded once per step.  The composite stencil
// reaches 6 nodes, so the CTA stages psi with ring 6, mu_psi on ring 4 and
// J_d on ring 2.
// ---------------------------------------------------------------------------
template <int TX, int TY> struct RKGeom {
    static constexpr int W6 = TX + 12, H6 = TY + 12;
    static constexpr int W4 = TX + 8, H4 = TY + 8;
    static constexpr int W2 = TX + 4, H2 = TY + 4;
    static constexpr int NSCALAR = W6 * H6 + W4 * H4 + 2 * W2 * H2;
    static_assert(W6 * H6 <= 2 * W2 * H2, "the d window fits the J arrays it precedes");
};

template <typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_rk_stage(KP<T> P, const T *__restrict__ phi, const T *__restrict__ din, const T *__restrict__ dbar,
           T *__restrict__ out, T a, T b, int last, T *__restrict__ philo)
{
    using G = RKGeom<TX, TY>;
    constexpr int W6 = G::W6, H6 = G::H6, W4 = G::W4, H4 = G::H4, W2 = G::W2, H2 = G::H2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_psi = reinterpret_cast<T *>(smem_raw);
    T *s_mu = s_psi + W6 * H6;
    T *s_jx = s_mu + W4 * H4;
    T *s_jy = s_jx + W2 * H2;
    T *s_d = s_jx;   // d window, consumed before J is written
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    load_tile<T, W6, H6>(s_psi, phi, x0 - 6, y0 - 6, P, false);
    load_tile<T, W6, H6>(s_d, din, x0 - 6, y0 - 6, P, false);
    tiles_ready();
    for (int t = threadIdx.x; t < W6 * H6; t += blockDim.x) s_psi[t] += s_d[t];
    __syncthreads();

    for (int t = threadIdx.x; t < W4 * H4; t += blockDim.x) {
        int ly = t / W4, lx = t - ly * W4;
        int i6 = (ly + 2) * W6 + (lx + 2);
        T v = s_psi[i6];
        T lap = fd4_d2<T, 1>(s_psi, i6) + fd4_d2<T, W6>(s_psi, i6);
        s_mu[t] = T(4) * P.beta * (v * v * v - v) - P.kappa * lap;
    }
    __syncthreads();

    for (int t = threadIdx.x; t < W2 * H2; t += blockDim.x) {
        int ly = t / W2, lx = t - ly * W2;
        int i6 = (ly + 4) * W6 + (lx + 4);
        int i4 = (ly + 2) * W4 + (lx + 2);
        T gx = fd4_d1<T, 1>(s_psi, i6), gy = fd4_d1<T, W6>(s_psi, i6);
        T v = s_psi[i6];
        const T m2 = gx * gx + gy * gy + P.eps2;
        const T inv = rsq(m2);
        const T mag = m2 * inv;
        T nxv = gx * inv, nyv = gy * inv;
        T jphi = mag - P.two_over_W * (T(1) - v * v);
        T jx = P.lambda * jphi * nxv, jy = P.lambda * jphi * nyv;
        if (P.flux_corr) {
            T mx = fd4_d1<T, 1>(s_mu, i4), my = fd4_d1<T, W4>(s_mu, i4);
            T dmn = mx * nxv + my * nyv;
            jx += -P.M * dmn * nxv;
            jy += -P.M * dmn * nyv;
        }
        s_jx[t] = jx;
        s_jy[t] = jy;
    }
    __syncthreads();

    for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
        int ly = t / TX, lx = t - ly * TX;
        const int X = x0 + lx, Y = y0 + ly;
        if (X >= P.nx || Y >= P.ny) continue;
        int i2 = (ly + 2) * W2 + (lx + 2);
        T L = fd4_d1<T, 1>(s_jx, i2) + fd4_d1<T, W2>(s_jy, i2);
        long long gidx = (long long)Y * P.nx + X;
        T r = b * (din[gidx] + L);
        if (a != T(0)) r = a * dbar[gidx] + r;
        if (last) {
            const T h = phi[gidx], s = h + r;
            if (philo) philo[gidx] = two_sum_err(h, r, s);
            r = s;
        }
        out[gidx] = r;
    }
}

// ---------------------------------------------------------------------------
// Pass 3: one Picard sweep of the implicit velocity (Sec. III.B Eq. u)
//   u^{k+1} = j + F(u^k) / (2 rho),
// F as in pass 1 but with phi^{n+1} and p_hat, the velocity gradients taken
// from the previous iterate u^k.
// ---------------------------------------------------------------------------
template <int TX, int TY> struct PCGeom {
    static constexpr int W2 = TX + 4, H2 = TY + 4;
    static constexpr int W1 = TX + 2, H1 = TY + 2;
    static constexpr int NSCALAR = W2 * H2 + 6 * W1 * H1;
};

// With gpop (the step's post-stream NS populations, [9][N]) the strain rate
// grad u + grad u^T of F_nu comes from their non-equilibrium part instead of
// the isotropic stencils (Sec. III.B Eq. Fmu, read for g):
//   S = [(s_7 - s_1)(F0.u) I - s_7 (F0 u + u F0)] / (2 rho cs^2)
//       - sum_i c_i c_i [M^-1 S^g M (g - g_eq(p_hat, u^k))]_i / cs^2,
// F0 being this sweep's force without F_nu.
template <typename T, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT)
k_picard(KP<T> P, const T *__restrict__ phi, const T *__restrict__ phat,
         const T *__restrict__ jx, const T *__restrict__ jy,
         const T *__restrict__ ukx, const T *__restrict__ uky,
         T *__restrict__ uox, T *__restrict__ uoy, const T *__restrict__ gpop)
{
    using G = PCGeom<TX, TY>;
    constexpr int W2 = G::W2, H2 = G::H2, W1 = G::W1, H1 = G::H1, A1 = W1 * H1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_phi = reinterpret_cast<T *>(smem_raw);
    T *s_p = s_phi + W2 * H2;
    T *s_ux = s_p + A1;
    T *s_uy = s_ux + A1;
    T *s_mu = s_uy + A1;
    T *s_gx = s_mu + A1;
    T *s_gy = s_gx + A1;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;

    load_tile<T, W2, H2>(s_phi, phi, x0 - 2, y0 - 2, P, false);
    load_tile<T, W1, H1>(s_p, phat, x0 - 1, y0 - 1, P, false);
    load_tile<T, W1, H1>(s_ux, ukx, x0 - 1, y0 - 1, P, true);
    load_tile<T, W1, H1>(s_uy, uky, x0 - 1, y0 - 1, P, true);
    tiles_ready();

    for (int t = threadIdx.x; t < A1; t += blockDim.x) {
        int ly = t / W1, lx = t - ly * W1;
        int i2 = (ly + 1) * W2 + (lx + 1);
        T ph = s_phi[i2];
        s_mu[t] = T(4) * P.beta * (ph * ph * ph - ph) - P.kappa * iso_lap<T, W2>(s_phi, i2);
        T gx, gy;
        iso_grad<T, W2>(s_phi, i2, gx, gy);
        s_gx[t] = gx;
        s_gy[t] = gy;
    }
    __syncthreads();

    for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
        int ly = t / TX, lx = t - ly * TX;
        const int X = x0 + lx, Y = y0 + ly;
        if (X >= P.nx || Y >= P.ny) continue;
        const long long gidx = (long long)Y * P.nx + X;
        const int i1 = (ly + 1) * W1 + (lx + 1);
        const T ph = s_phi[(ly + 2) * W2 + (lx + 2)];
        T rho, ir, nu;
        rho_nu(P, ph, rho, ir, nu);
        const T grx = P.drho * s_gx[i1], gry = P.drho * s_gy[i1];
        T dmx, dmy;
        iso_grad<T, W1>(s_mu, i1, dmx, dmy);
        const T Jx = P.drho * P.M * dmx, Jy = P.drho * P.M * dmy;
        T Fsx, Fsy;
        {
            const int nb[8] = {i1 + 1, i1 - 1, i1 + W1, i1 - W1, i1 + W1 + 1, i1 + W1 - 1, i1 - W1 - 1, i1 - W1 + 1};
            T txx[8], txy[8], tyy[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const T a = s_gx[nb[k]], b = s_gy[nb[k]];
                txx[k] = b * b;
                txy[k] = -a * b;
                tyy[k] = a * a;
            }
            const T dxx = (txx[0] - txx[1]) * T(1.0 / 3.0) + (txx[4] - txx[5] - txx[6] + txx[7]) * T(1.0 / 12.0);
            const T dyxy = (txy[2] - txy[3]) * T(1.0 / 3.0) + (txy[4] + txy[5] - txy[6] - txy[7]) * T(1.0 / 12.0);
            const T dxxy = (txy[0] - txy[1]) * T(1.0 / 3.0) + (txy[4] - txy[5] - txy[6] + txy[7]) * T(1.0 / 12.0);
            const T dyyy = (tyy[2] - tyy[3]) * T(1.0 / 3.0) + (tyy[4] + tyy[5] - tyy[6] - tyy[7]) * T(1.0 / 12.0);
            Fsx = P.kappa * (dxx + dyxy);
            Fsy = P.kappa * (dxxy + dyyy);
        }
        const T pc = s_p[i1];
        T dxux, dyux, dxuy, dyuy;
        iso_grad<T, W1>(s_ux, i1, dxux, dyux);
        iso_grad<T, W1>(s_uy, i1, dxuy, dyuy);
        T Sxx = T(2) * dxux, Sxy = dyux + dxuy, Syy = T(2) * dyuy;
        const T F0x = -pc * grx + Fsx + (Jx * dxux + Jy * dyux) + (rho - P.g_rho_ref) * P.gx;
        const T F0y = -pc * gry + Fsy + (Jx * dxuy + Jy * dyuy) + (rho - P.g_rho_ref) * P.gy;
        if (gpop) {   // strain rate from the non-equilibrium moments
            const T u0 = s_ux[i1], u1 = s_uy[i1];
            constexpr int cxv[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
            constexpr int cyv[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
            const T u2 = u0 * u0 + u1 * u1;
            T d[9], m[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const T cu = T(cxv[q]) * u0 + T(cyv[q]) * u1;
                const T geq = lattice_w_t<T>(q) * (T(3) * pc + T(3) * cu + T(4.5) * cu * cu - T(1.5) * u2);
                d[q] = gpop[(size_t)gidx + (size_t)q * P.N] - geq;
            }
            to_moments(d, m);
            const T s78 = rcp(nu * T(3) + T(0.5));
#pragma unroll
            for (int k = 0; k < 9; ++k) m[k] *= k < 7 ? P.sg[k] : s78;
            from_moments(m, d);
            T pxx = T(0), pxy = T(0), pyy = T(0);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                pxx += T(cxv[q] * cxv[q]) * d[q];
                pxy += T(cxv[q] * cyv[q]) * d[q];
                pyy += T(cyv[q] * cyv[q]) * d[q];
            }
            const T Fu = F0x * u0 + F0y * u1, a = T(1.5) * ir;   // 1 / (2 rho cs^2)
            Sxx = ((s78 - P.sg[1]) * Fu - s78 * T(2) * F0x * u0) * a - T(3) * pxx;
            Sxy = -s78 * (F0x * u1 + u0 * F0y) * a - T(3) * pxy;
            Syy = ((s78 - P.sg[1]) * Fu - s78 * T(2) * F0y * u1) * a - T(3) * pyy;
        }
        const T Fx = F0x + nu * (Sxx * grx + Sxy * gry);
        const T Fy = F0y + nu * (Sxy * grx + Syy * gry);
        const T h = T(0.5) * ir;
        uox[gidx] = jx[gidx] + Fx * h;
        uoy[gidx] = jy[gidx] + Fy * h;
    }
}

// ---------------------------------------------------------------------------
// Pass 4: explicit selective filter (Sec. III.B Eq. filter, App. B) of
// chi = (p, ux, uy), every node from the unfiltered field:
//   chi <- chi - a [ 2 d_0 chi + sum_{m=1..R} d_m (chi_{x+m} + chi_{x-m} + chi_{y+m} + chi_{y-m}) ].
// ---------------------------------------------------------------------------
template <int TX, int TY, int R> struct FLGeom {
    static constexpr int WR = TX + 2 * R, HR = TY + 2 * R;
    static constexpr int NSCALAR = 3 * WR * HR;
};

template <typename T, int TX, int TY, int R, int NT>
__global__ void __launch_bounds__(NT)
k_filter(KP<T> P, const T *__restrict__ pin, const T *__restrict__ uxin, const T *__restrict__ uyin,
         T *__restrict__ pout, T *__restrict__ uxout, T *__restrict__ uyout)
{
    using G = FLGeom<TX, TY, R>;
    constexpr int WR = G::WR, HR = G::HR, A = WR * HR;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_p = reinterpret_cast<T *>(smem_raw);
    T *s_ux = s_p + A;
    T *s_uy = s_ux + A;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    load_tile<T, WR, HR>(s_p, pin, x0 - R, y0 - R, P, false);
    load_tile<T, WR, HR>(s_ux, uxin, x0 - R, y0 - R, P, true);
    load_tile<T, WR, HR>(s_uy, uyin, x0 - R, y0 - R, P, true);
    tiles_ready();
    for (int t = threadIdx.x; t < TX * TY; t += blockDim.x) {
        int ly = t / TX, lx = t - ly * TX;
        const int X = x0 + lx, Y = y0 + ly;
        if (X >= P.nx || Y >= P.ny) continue;
        const long long gidx = (long long)Y * P.nx + X;
        const int c = (ly + R) * WR + (lx + R);
        T *arr[3] = {s_p, s_ux, s_uy};
        T res[3];
#pragma unroll
        for (int v = 0; v < 3; ++v) {
            const T *s = arr[v];
            T acc = T(2) * P.fd[0] * s[c];
#pragma unroll
            for (int m = 1; m <= R; ++m)
                acc += P.fd[m] * (s[c + m] + s[c - m] + s[c + m * WR] + s[c - m * WR]);
            res[v] = s[c] - P.fa * acc;
        }
        pout[gidx] = res[0];
        uxout[gidx] = res[1];
        uyout[gidx] = res[2];
    }
}

// Paired FP32 arithmetic: two horizontally adjacent nodes per thread, so that
// the additions and multiply-adds issue as FADD2 / FFMA2 on float2 operands.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Filtered values of one field at the column pair (X, X+1) over VR rows from
// ly0, the window s of row stride WR holding the field from column X - RP.
template <int WR, int R, int VR>
__device__ __forceinline__ void filter_strip(const KP<float> &P, const float *sv, int lx, int ly0, int y0, int X,
                                             float *__restrict__ out)
{
    constexpr int RP = (R + 1) & ~1;
    const float2 na = f2(-P.fa);
    float2 col[VR + 2 * R];   // rows ly0 - R .. ly0 + VR - 1 + R of columns (X, X+1)
#pragma unroll
    for (int k = 0; k < VR + 2 * R; ++k)
        col[k] = *reinterpret_cast<const float2 *>(&sv[(ly0 + k) * WR + lx + RP]);
#pragma unroll
    for (int i = 0; i < VR; ++i) {
        const int Y = y0 + ly0 + i;
        if (Y >= P.ny) break;
        const int c = (ly0 + R + i) * WR + lx + RP;
        float2 w[RP + 1];
#pragma unroll
        for (int k = 0; k < RP + 1; ++k) w[k] = *reinterpret_cast<const float2 *>(&sv[c - RP + 2 * k]);
        const float2 ctr = col[R + i];
        float2 acc = mul2(f2(2.0f * P.fd[0]), ctr);
#pragma unroll
        for (int m = 1; m <= R; ++m) {
            const int e0 = RP + m, e1 = RP + m + 1, w0 = RP - m, w1 = RP - m + 1;
            const float ex0 = (e0 & 1) ? w[e0 >> 1].y : w[e0 >> 1].x;
            const float ex1 = (e1 & 1) ? w[e1 >> 1].y : w[e1 >> 1].x;
            const float wx0 = (w0 & 1) ? w[w0 >> 1].y : w[w0 >> 1].x;
            const float wx1 = (w1 & 1) ? w[w1 >> 1].y : w[w1 >> 1].x;
            // even m: whole register pairs; odd m: pairs straddle, scalar sums
            float2 sum = (m & 1) ? make_float2(ex0 + wx0, ex1 + wx1) : add2(w[e0 >> 1], w[w0 >> 1]);
            sum = add2(sum, add2(col[R + i + m], col[R + i - m]));
            acc = fma2(f2(P.fd[m]), sum, acc);
        }
        *reinterpret_cast<float2 *>(&out[(long long)Y * P.nx + X]) = fma2(na, acc, ctr);
    }
}

// Filter pass for FP32 on grids of even width, with register reuse: each
// thread filters a 2-column x VR-row block.  The y-taps of the whole block
// come from one column of VR + 2R aligned float2 reads held in registers; the
// x-taps of each row from RP + 1 aligned float2 reads.
// The three filtered fields of a TX x TY tile, thread t on the column pair
// 2 (t mod TX/2) over VR rows; the windows hold the fields from
// (x0 - RP, y0 - R) with row stride SW.
template <int TX, int TY, int R, int VR, int SW>
__device__ __forceinline__ void filter_strips_body(const KP<float> &P, const float *s_p, const float *s_ux,
                                                   const float *s_uy, int x0, int y0, float *__restrict__ pout,
                                                   float *__restrict__ uxout, float *__restrict__ uyout)
{
    const int t = threadIdx.x;
    const int lx = 2 * (t % (TX / 2)), ly0 = (t / (TX / 2)) * VR;
    const int X = x0 + lx;
    if (X >= P.nx) return;
    filter_strip<SW, R, VR>(P, s_p, lx, ly0, y0, X, pout);
    filter_strip<SW, R, VR>(P, s_ux, lx, ly0, y0, X, uxout);
    filter_strip<SW, R, VR>(P, s_uy, lx, ly0, y0, X, uyout);
}

template <int TX, int TY, int R, int VR> struct FLSGeom {
    static constexpr int RP = (R + 1) & ~1;
    static constexpr int WR = TX + 2 * RP, HR = TY + 2 * R;
    static constexpr int NT = (TX / 2) * (TY / VR);
    static constexpr int NSCALAR = 3 * WR * HR;
};

template <int TX, int TY, int R, int VR>
__global__ void __launch_bounds__((TX / 2) * (TY / VR), 3)
k_filter_strips(KP<float> P, const float *__restrict__ pin, const float *__restrict__ uxin,
                const float *__restrict__ uyin, float *__restrict__ pout, float *__restrict__ uxout,
                float *__restrict__ uyout)
{
    using G = FLSGeom<TX, TY, R, VR>;
    constexpr int RP = G::RP, WR = G::WR, HR = G::HR, A = WR * HR;
    static_assert(TX % 2 == 0 && WR % 2 == 0 && TY % VR == 0, "pairs need even widths");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_p = reinterpret_cast<float *>(smem_raw);
    float *s_ux = s_p + A;
    float *s_uy = s_ux + A;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    load_tile<float, WR, HR>(s_p, pin, x0 - RP, y0 - R, P, false);
    load_tile<float, WR, HR>(s_ux, uxin, x0 - RP, y0 - R, P, true);
    load_tile<float, WR, HR>(s_uy, uyin, x0 - RP, y0 - R, P, true);
    tiles_ready();
    filter_strips_body<TX, TY, R, VR, WR>(P, s_p, s_ux, s_uy, x0, y0, pout, uxout, uyout);
}

// Fourth-order differences (Sec. III.A Eq. fourOrder_FDM) of the node pair
// (x, x+1), x even, from the aligned pairs l = (x-2, x-1), c = (x, x+1),
// r = (x+2, x+3) of a row, or from five rows of pairs (y-derivatives).
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return fma2(f2(-1.0f), b, a); }
__device__ __forceinline__ float2 pd1(float2 m2, float2 m1, float2 p1, float2 p2)
{
    return fma2(f2(2.0f / 3.0f), sub2(p1, m1), mul2(f2(1.0f / 12.0f), sub2(m2, p2)));
}
__device__ __forceinline__ float2 pd2(float2 m2, float2 m1, float2 c, float2 p1, float2 p2)
{
    return fma2(f2(4.0f / 3.0f), add2(m1, p1), fma2(f2(-2.5f), c, mul2(f2(-1.0f / 12.0f), add2(m2, p2))));
}
// (the neighbours at distance 1 straddle register pairs: their difference
// and sum are formed in scalar arithmetic)
__device__ __forceinline__ float2 pd1x(float2 l, float2 c, float2 r)
{
    return fma2(f2(2.0f / 3.0f), make_float2(c.y - l.y, r.x - c.x), mul2(f2(1.0f / 12.0f), sub2(l, r)));
}
__device__ __forceinline__ float2 pd2x(float2 l, float2 c, float2 r)
{
    return fma2(f2(4.0f / 3.0f), make_float2(l.y + c.y, c.x + r.x),
                fma2(f2(-2.5f), c, mul2(f2(-1.0f / 12.0f), add2(l, r))));
}
#ifdef LBM_DEBUG
// Debug builds (LBM_DEBUG) check every paired shared-memory access of the
// FP32 kernels (lds2/sts2 on a pointer into shared memory; sts2 also
// stores to global planes, which are not checked) against the launch's
// dynamic shared memory.  An access outside it is not made (a load returns
// zero) and the first one is recorded in g_lbm_debug: the block index in
// the high 32 bits, 1 + the byte offset from the start of the dynamic
// shared memory (two's complement, low 31 bits) in the low ones.
static __device__ unsigned long long g_lbm_debug;
extern __shared__ __align__(16) unsigned char lbm_dyn_smem[];
__device__ __forceinline__ bool smem_in(const float *s, int i)
{
    if (!__isShared(s)) return true;   // a global plane
    unsigned dyn;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const long long off = (long long)(reinterpret_cast<const unsigned char *>(s + i) - lbm_dyn_smem);
    if (off >= 0 && off + 8 <= (long long)dyn) return true;
    const unsigned long long blk = blockIdx.x + (unsigned long long)gridDim.x * blockIdx.y;
    atomicCAS(&g_lbm_debug, 0ull, (blk << 32) | (((unsigned long long)off & 0x7fffffffull) + 1ull));
    return false;
}
__device__ __forceinline__ float2 lds2(const float *s, int i)
{
    return smem_in(s, i) ? *reinterpret_cast<const float2 *>(s + i) : make_float2(0.0f, 0.0f);
}
#else
__device__ __forceinline__ float2 lds2(const float *s, int i) { return *reinterpret_cast<const float2 *>(s + i); }
#endif
// phi^{n+1} = phi_hi + r for the pair: returns the new phi_hi and writes the
// new phi_lo to *lo.
__device__ __forceinline__ float2 add_hi_lo(float2 h, float2 r, float *lo)
{
    const float2 s = make_float2(__fadd_rn(h.x, r.x), __fadd_rn(h.y, r.y));
    *reinterpret_cast<float2 *>(lo) = make_float2(two_sum_err(h.x, r.x, s.x), two_sum_err(h.y, r.y, s.y));
    return s;
}
#ifdef LBM_DEBUG
__device__ __forceinline__ void sts2(float *s, int i, float2 v)
{
    if (smem_in(s, i)) *reinterpret_cast<float2 *>(s + i) = v;
}
#else
__device__ __forceinline__ void sts2(float *s, int i, float2 v) { *reinterpret_cast<float2 *>(s + i) = v; }
#endif

// Item it of a region of NP column pairs by NB bands of rows, numbered so
// that the lanes of a warp share a band: the first 32 pairs of every band
// come first, a band per 32 items, then the remaining NP - 32 pairs of every
// band.  (Numbered row-major instead, a warp whose items straddle two bands
// reads shared-memory rows that fall on the same banks.)
template <int NP, int NB> __device__ __forceinline__ void band_item(int it, int &pair, int &band)
{
    constexpr int MAIN = NP < 32 ? NP : 32, REST = NP - MAIN;
    if (REST == 0 || it < MAIN * NB) {
        band = it / MAIN;
        pair = it - band * MAIN;
    } else {
        const int j = it - MAIN * NB;
        band = j / (REST > 0 ? REST : 1);
        pair = MAIN + j - band * REST;
    }
}

// Pass 2 for FP32 on grids of even width, same tile and result as
// k_rk_stage: each thread covers a column pair over VR1 / VR2 / VR3 rows of
// the mu / J / divergence regions, holding the y-neighbours in registers.
// s_psi holds psi from (x0 - 6, y0 - 6) with row stride SW.
// emit(i, gidx, L) receives L(psi) at row i of the thread's output strip
// (global index gidx of its first column) and writes the stage's result.
template <int TX, int TY, int NT, int VR1, int VR2, int VR3, int SW, typename EMIT>
__device__ __forceinline__ void rk_strips_body(const KP<float> &P, const float *s_psi, float *s_mu, float *s_jx,
                                               float *s_jy, int x0, int y0, EMIT &&emit)
{
    using G = RKGeom<TX, TY>;
    constexpr int W4 = G::W4, H4 = G::H4, W2 = G::W2, H2 = G::H2;
    static_assert(TX % 2 == 0 && SW % 2 == 0 && H4 % VR1 == 0 && H2 % VR2 == 0 && TY % VR3 == 0,
                  "strips must tile the regions");

    if (P.flux_corr) {   // mu on the (TX+8) x (TY+8) region, psi offset 2
        constexpr int NP = W4 / 2, NB = H4 / VR1, NI = NP * NB;
        const float2 fb = f2(4.0f * P.beta), nk = f2(-P.kappa);
        for (int it = threadIdx.x; it < NI; it += NT) {
            int pr, bd;
            band_item<NP, NB>(it, pr, bd);
            const int lx = 2 * pr, r0 = bd * VR1;
            const int xc = lx + 2;
            float2 w[VR1 + 4];
#pragma unroll
            for (int k = 0; k < VR1 + 4; ++k) w[k] = lds2(s_psi, (r0 + k) * SW + xc);
#pragma unroll
            for (int i = 0; i < VR1; ++i) {
                const int row = (r0 + 2 + i) * SW + xc;
                const float2 c = w[i + 2];
                const float2 lap = add2(pd2x(lds2(s_psi, row - 2), c, lds2(s_psi, row + 2)),
                                        pd2(w[i], w[i + 1], c, w[i + 3], w[i + 4]));
                const float2 c3 = mul2(mul2(c, c), c);
                sts2(s_mu, (r0 + i) * W4 + lx, fma2(fb, sub2(c3, c), mul2(nk, lap)));
            }
        }
        __syncthreads();
    }

    {   // J = lambda J_phi n + q on the (TX+4) x (TY+4) region, psi offset 4, mu offset 2
        constexpr int NP = W2 / 2, NB = H2 / VR2, NI = NP * NB;
        const float2 lam = f2(P.lambda), tw = f2(P.two_over_W), e2 = f2(P.eps2), nm = f2(-P.M);
        for (int it = threadIdx.x; it < NI; it += NT) {
            int pr, bd;
            band_item<NP, NB>(it, pr, bd);
            const int lx = 2 * pr, r0 = bd * VR2;
            const int xc = lx + 4;
            float2 w[VR2 + 4];
#pragma unroll
            for (int k = 0; k < VR2 + 4; ++k) w[k] = lds2(s_psi, (r0 + 2 + k) * SW + xc);
            float2 wm[VR2 + 4];
            if (P.flux_corr) {
#pragma unroll
                for (int k = 0; k < VR2 + 4; ++k) wm[k] = lds2(s_mu, (r0 + k) * W4 + lx + 2);
            }
#pragma unroll
            for (int i = 0; i < VR2; ++i) {
                const int row = (r0 + 4 + i) * SW + xc;
                const float2 v = w[i + 2];
                const float2 gx = pd1x(lds2(s_psi, row - 2), v, lds2(s_psi, row + 2));
                const float2 gy = pd1(w[i], w[i + 1], w[i + 3], w[i + 4]);
                const float2 m2 = fma2(gx, gx, fma2(gy, gy, e2));
                const float2 inv = make_float2(rsqrtf(m2.x), rsqrtf(m2.y));
                const float2 nx = mul2(gx, inv), ny = mul2(gy, inv);
                // |grad psi| - (2/W)(1 - psi^2)
                const float2 jphi = fma2(tw, fma2(v, v, f2(-1.0f)), mul2(m2, inv));
                const float2 lj = mul2(lam, jphi);
                float2 jx = mul2(lj, nx), jy = mul2(lj, ny);
                if (P.flux_corr) {
                    const int mrow = (r0 + 2 + i) * W4 + lx + 2;
                    const float2 mx = pd1x(lds2(s_mu, mrow - 2), wm[i + 2], lds2(s_mu, mrow + 2));
                    const float2 my = pd1(wm[i], wm[i + 1], wm[i + 3], wm[i + 4]);
                    const float2 t = mul2(nm, fma2(mx, nx, mul2(my, ny)));
                    jx = fma2(t, nx, jx);
                    jy = fma2(t, ny, jy);
                }
                sts2(s_jx, (r0 + i) * W2 + lx, jx);
                sts2(s_jy, (r0 + i) * W2 + lx, jy);
            }
        }
    }
    __syncthreads();

    {   // div J on the tile, J offset 2
        constexpr int NP = TX / 2, NI = NP * (TY / VR3);
        for (int it = threadIdx.x; it < NI; it += NT) {
            const int lx = 2 * (it % NP), r0 = (it / NP) * VR3;
            const int X = x0 + lx;
            if (X >= P.nx) continue;
            float2 w[VR3 + 4];
#pragma unroll
            for (int k = 0; k < VR3 + 4; ++k) w[k] = lds2(s_jy, (r0 + k) * W2 + lx + 2);
#pragma unroll
            for (int i = 0; i < VR3; ++i) {
                const int Y = y0 + r0 + i;
                if (Y >= P.ny) break;
                const int jrow = (r0 + 2 + i) * W2 + lx + 2;
                const float2 L = add2(pd1x(lds2(s_jx, jrow - 2), lds2(s_jx, jrow), lds2(s_jx, jrow + 2)),
                                      pd1(w[i], w[i + 1], w[i + 3], w[i + 4]));
                emit(i, (long long)Y * P.nx + X, L);
            }
        }
    }
}

template <int TX, int TY, int NT, int VR1, int VR2, int VR3>
__global__ void __launch_bounds__(NT, 3)
k_rk_strips(KP<float> P, const float *__restrict__ phi, const float *__restrict__ din,
            const float *__restrict__ dbar, float *__restrict__ out, float a, float b, int last,
            float *__restrict__ philo)
{
    using G = RKGeom<TX, TY>;
    constexpr int W6 = G::W6, H6 = G::H6, W4 = G::W4, H4 = G::H4, W2 = G::W2, H2 = G::H2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_psi = reinterpret_cast<float *>(smem_raw);
    float *s_mu = s_psi + W6 * H6;
    float *s_jx = s_mu + W4 * H4;
    float *s_jy = s_jx + W2 * H2;
    float *s_d = s_jx;   // d window, consumed before J is written
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    load_tile<float, W6, H6>(s_psi, phi, x0 - 6, y0 - 6, P, false);
    load_tile<float, W6, H6>(s_d, din, x0 - 6, y0 - 6, P, false);
    tiles_ready();
    for (int t = threadIdx.x; t < W6 * H6; t += NT) s_psi[t] += s_d[t];
    __syncthreads();
    const float2 aa = f2(a), bb = f2(b);
    rk_strips_body<TX, TY, NT, VR1, VR2, VR3, W6>(
        P, s_psi, s_mu, s_jx, s_jy, x0, y0, [&](int, long long gidx, float2 L) {
            float2 r = mul2(bb, add2(*reinterpret_cast<const float2 *>(&din[gidx]), L));
            if (a != 0.0f) r = fma2(aa, *reinterpret_cast<const float2 *>(&dbar[gidx]), r);
            if (last) r = add_hi_lo(*reinterpret_cast<const float2 *>(&phi[gidx]), r, philo + gidx);
            *reinterpret_cast<float2 *>(&out[gidx]) = r;
        });
}

// Pass 3 for FP32 on grids of even width, same result as k_picard: each
// thread covers a column pair over VR2 rows.  Of each row of a 3 x 3
// neighbourhood only D = E - W and U = C/3 + (E + W)/12 are kept, from which
// the isotropic derivatives of Sec. III.B Eq. dicretized follow as
//   d_x = D_0 / 3 + (D_+ + D_-) / 12,   d_y = U_+ - U_-.
template <int TX, int TY> struct PSGeom {
    static constexpr int WP = TX + 8, HP = TY + 4;   // phi, origin (x0 - 4, y0 - 2)
    static constexpr int WA = TX + 4, HA = TY + 2;   // p, u, mu, grad phi, origin (x0 - 2, y0 - 1)
    static constexpr int NSCALAR = WP * HP + 6 * WA * HA;
};

// The x-neighbours of the pair, (l.y, c.x) and (c.y, r.x), straddle register
// pairs: their difference and sum are formed in scalar arithmetic, which
// costs less than assembling the pairs for FADD2.
__device__ __forceinline__ void iso_row(float2 l, float2 c, float2 r, float2 &D, float2 &U)
{
    D = make_float2(c.y - l.y, r.x - c.x);
    const float2 S = make_float2(c.y + l.y, r.x + c.x);
    U = fma2(f2(1.0f / 3.0f), c, mul2(f2(1.0f / 12.0f), S));
}
__device__ __forceinline__ float2 iso_dx(float2 Ds, float2 Dc, float2 Dn)
{
    return fma2(f2(1.0f / 3.0f), Dc, mul2(f2(1.0f / 12.0f), add2(Dn, Ds)));
}

struct PicardRow {
    float2 Dm, Um;              // mu
    float2 Dxx, Dxy, Uxy, Uyy;  // T = (gy^2, -gx gy; -gx gy, gx^2)
    float2 Dux, Uux, Duy, Uuy;  // u^k
};

// mu and grad phi of Sec. III.B Eq. dicretized over a region of NPA column
// pairs x NRA rows (strips of VR1 rows).  s_phi points at the region's origin
// less two columns and one row, with row stride SP; the outputs have row
// stride WA from the region's origin.
template <int NPA, int NRA, int VR1, int NT, int SP, int WA>
__device__ __forceinline__ void picard_mu_grad(const KP<float> &P, const float *s_phi, float *s_mu, float *s_gx,
                                               float *s_gy)
{
    static_assert(NRA % VR1 == 0 && SP % 2 == 0 && WA % 2 == 0, "strips must tile the region");
    constexpr int NB = NRA / VR1, NI = NPA * NB;
    const float2 fb = f2(4.0f * P.beta), nk = f2(-P.kappa);
    for (int it = threadIdx.x; it < NI; it += NT) {
        int pr, bd;
        band_item<NPA, NB>(it, pr, bd);
        const int lx = 2 * pr, r0 = bd * VR1;
        float2 C[VR1 + 2], D[VR1 + 2], S[VR1 + 2];
#pragma unroll
        for (int k = 0; k < VR1 + 2; ++k) {
            const int row = (r0 + k) * SP + lx + 2;
            const float2 l = lds2(s_phi, row - 2), c = lds2(s_phi, row), r = lds2(s_phi, row + 2);
            C[k] = c;
            D[k] = make_float2(c.y - l.y, r.x - c.x);
            S[k] = make_float2(c.y + l.y, r.x + c.x);
        }
#pragma unroll
        for (int i = 0; i < VR1; ++i) {
            const float2 gx = iso_dx(D[i], D[i + 1], D[i + 2]);
            const float2 gy = fma2(f2(1.0f / 3.0f), sub2(C[i + 2], C[i]), mul2(f2(1.0f / 12.0f), sub2(S[i + 2], S[i])));
            const float2 lap = fma2(f2(2.0f / 3.0f), add2(S[i + 1], add2(C[i + 2], C[i])),
                                    fma2(f2(1.0f / 6.0f), add2(S[i + 2], S[i]), mul2(f2(-10.0f / 3.0f), C[i + 1])));
            const float2 ph = C[i + 1];
            const float2 mu = fma2(fb, sub2(mul2(mul2(ph, ph), ph), ph), mul2(nk, lap));
            const int o = (r0 + i) * WA + lx;
            sts2(s_mu, o, mu);
            sts2(s_gx, o, gx);
            sts2(s_gy, o, gy);
        }
    }
}

// One Picard sweep, u^{k+1} = j + F(u^k) / (2 rho) (Sec. III.B), over a
// region of NP column pairs x NR rows with global origin (X0, Y0), in strips
// of VR2 rows.  s_mu, s_gx, s_gy (row stride WA) and s_p, s_ux, s_uy (row
// stride SA) point at the region's origin less two columns and one row;
// s_phi (row stride SP) at the origin less four columns and two rows.  With
// CLIP, pairs and rows outside the domain are skipped (an output region);
// without, every node of the region is computed (a ring around a tile,
// whose inputs were staged through the wrap/mirror map).
// jf(i, ly, lx, X, Y, jx, jy) returns j at row i of the thread's strip
// (region row ly, column lx, global X, Y); out(i, ly, lx, X, Y, ux, uy)
// receives u^{k+1} there.
template <int NP, int NR, int VR2, int NT, int WA, int SA, int SP, bool CLIP, typename JF, typename OUT>
__device__ __forceinline__ void picard_sweep(const KP<float> &P, const float *s_mu, const float *s_gx,
                                             const float *s_gy, const float *s_p, const float *s_ux,
                                             const float *s_uy, const float *s_phi, int X0, int Y0, JF &&jf,
                                             OUT &&out)
{
    static_assert(NR % VR2 == 0 && WA % 2 == 0 && SA % 2 == 0 && SP % 2 == 0, "strips must tile the region");
    constexpr int NI = NP * (NR / VR2);
    const float2 dr = f2(P.drho), drm = f2(P.drho * P.M), kap = f2(P.kappa);
    for (int it = threadIdx.x; it < NI; it += NT) {
        const int lx = 2 * (it % NP), r0 = (it / NP) * VR2;
        const int X = X0 + lx;
        if (CLIP && X >= P.nx) continue;
        PicardRow rw[VR2 + 2];
#pragma unroll
        for (int k = 0; k < VR2 + 2; ++k) {
            const int a = (r0 + k) * WA + lx + 2, au = (r0 + k) * SA + lx + 2;
            iso_row(lds2(s_mu, a - 2), lds2(s_mu, a), lds2(s_mu, a + 2), rw[k].Dm, rw[k].Um);
            const float2 gxl = lds2(s_gx, a - 2), gxc = lds2(s_gx, a), gxr = lds2(s_gx, a + 2);
            const float2 gyl = lds2(s_gy, a - 2), gyc = lds2(s_gy, a), gyr = lds2(s_gy, a + 2);
            float2 dummy;
            iso_row(mul2(gyl, gyl), mul2(gyc, gyc), mul2(gyr, gyr), rw[k].Dxx, dummy);
            const float2 m1 = f2(-1.0f);
            iso_row(mul2(m1, mul2(gxl, gyl)), mul2(m1, mul2(gxc, gyc)), mul2(m1, mul2(gxr, gyr)), rw[k].Dxy,
                    rw[k].Uxy);
            iso_row(mul2(gxl, gxl), mul2(gxc, gxc), mul2(gxr, gxr), dummy, rw[k].Uyy);
            iso_row(lds2(s_ux, au - 2), lds2(s_ux, au), lds2(s_ux, au + 2), rw[k].Dux, rw[k].Uux);
            iso_row(lds2(s_uy, au - 2), lds2(s_uy, au), lds2(s_uy, au + 2), rw[k].Duy, rw[k].Uuy);
            if (k < 2) continue;
            // output row i = k - 2 from rows k - 2 (south), k - 1 (centre), k (north)
            const int i = k - 2;
            const int Y = Y0 + r0 + i;
            if (CLIP && Y >= P.ny) break;
            const PicardRow &sR = rw[k - 2], &cR = rw[k - 1], &nR = rw[k];
            const float2 dmx = iso_dx(sR.Dm, cR.Dm, nR.Dm), dmy = sub2(nR.Um, sR.Um);
            const float2 Fsx = mul2(kap, add2(iso_dx(sR.Dxx, cR.Dxx, nR.Dxx), sub2(nR.Uxy, sR.Uxy)));
            const float2 Fsy = mul2(kap, add2(iso_dx(sR.Dxy, cR.Dxy, nR.Dxy), sub2(nR.Uyy, sR.Uyy)));
            const float2 dxux = iso_dx(sR.Dux, cR.Dux, nR.Dux), dyux = sub2(nR.Uux, sR.Uux);
            const float2 dxuy = iso_dx(sR.Duy, cR.Duy, nR.Duy), dyuy = sub2(nR.Uuy, sR.Uuy);
            const int ac = (r0 + i + 1) * WA + lx + 2;
            const float2 grx = mul2(dr, lds2(s_gx, ac)), gry = mul2(dr, lds2(s_gy, ac));
            const float2 Jx = mul2(drm, dmx), Jy = mul2(drm, dmy);
            const float2 pc = lds2(s_p, (r0 + i + 1) * SA + lx + 2);
            const float2 ph = lds2(s_phi, (r0 + i + 2) * SP + lx + 4);
            float2 rho, ir, nu;
            rho_nu(P, ph.x, rho.x, ir.x, nu.x);
            rho_nu(P, ph.y, rho.y, ir.y, nu.y);
            const float2 Sxx = add2(dxux, dxux), Sxy = add2(dyux, dxuy), Syy = add2(dyuy, dyuy);
            const float2 rg = sub2(rho, f2(P.g_rho_ref));
            float2 Fx = fma2(rg, f2(P.gx), fma2(Jx, dxux, mul2(Jy, dyux)));
            float2 Fy = fma2(rg, f2(P.gy), fma2(Jx, dxuy, mul2(Jy, dyuy)));
            Fx = fma2(nu, fma2(Sxx, grx, mul2(Sxy, gry)), add2(Fx, fma2(mul2(m1, pc), grx, Fsx)));
            Fy = fma2(nu, fma2(Sxy, grx, mul2(Syy, gry)), add2(Fy, fma2(mul2(m1, pc), gry, Fsy)));
            const float2 hh = mul2(f2(0.5f), ir);
            float2 jxv, jyv;
            jf(i, r0 + i, lx, X, Y, jxv, jyv);
            out(i, r0 + i, lx, X, Y, fma2(Fx, hh, jxv), fma2(Fy, hh, jyv));
        }
    }
}

// s_phi holds phi from (x0 - 4, y0 - 2) with row stride SP; s_p, s_ux, s_uy
// hold p_hat, u^k from (x0 - 2, y0 - 1) with row stride SA; s_mu, s_gx, s_gy
// are (TX + 4) x (TY + 2) work arrays.
// jf(i, ly, lx, gidx, jx, jy) returns j at row i of the thread's strip (tile
// row ly), column pair lx (global index gidx).
template <int TX, int TY, int NT, int VR1, int VR2, int SP, int SA, typename JF>
__device__ __forceinline__ void picard_strips_body(const KP<float> &P, const float *s_phi, const float *s_p,
                                                   const float *s_ux, const float *s_uy, float *s_mu, float *s_gx,
                                                   float *s_gy, int x0, int y0, JF &&jf, float *__restrict__ uox,
                                                   float *__restrict__ uoy)
{
    using G = PSGeom<TX, TY>;
    constexpr int WA = G::WA, HA = G::HA;
    static_assert(TX % 2 == 0 && SP % 2 == 0 && SA % 2 == 0 && HA % VR1 == 0 && TY % VR2 == 0,
                  "strips must tile the regions");
    // mu and grad phi on the (TX+4) x (TY+2) region
    picard_mu_grad<WA / 2, HA, VR1, NT, SP, WA>(P, s_phi, s_mu, s_gx, s_gy);
    __syncthreads();
    // u^{k+1} = j + F(u^k) / (2 rho) on the tile
    picard_sweep<TX / 2, TY, VR2, NT, WA, SA, SP, true>(
        P, s_mu, s_gx, s_gy, s_p, s_ux, s_uy, s_phi, x0, y0,
        [&](int i, int ly, int lx, int X, int Y, float2 &a, float2 &b) {
            jf(i, ly, lx, (long long)Y * P.nx + X, a, b);
        },
        [&](int, int, int, int X, int Y, float2 vx, float2 vy) {
            const long long gidx = (long long)Y * P.nx + X;
            *reinterpret_cast<float2 *>(&uox[gidx]) = vx;
            *reinterpret_cast<float2 *>(&uoy[gidx]) = vy;
        });
}

template <int TX, int TY, int NT, int VR1, int VR2>
__global__ void __launch_bounds__(NT, 3)
k_picard_strips(KP<float> P, const float *__restrict__ phi, const float *__restrict__ phat,
                const float *__restrict__ jx, const float *__restrict__ jy,
                const float *__restrict__ ukx, const float *__restrict__ uky,
                float *__restrict__ uox, float *__restrict__ uoy)
{
    using G = PSGeom<TX, TY>;
    constexpr int WP = G::WP, HP = G::HP, WA = G::WA, HA = G::HA, AA = WA * HA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *s_phi = reinterpret_cast<float *>(smem_raw);
    float *s_p = s_phi + WP * HP;
    float *s_ux = s_p + AA;
    float *s_uy = s_ux + AA;
    float *s_mu = s_uy + AA;
    float *s_gx = s_mu + AA;
    float *s_gy = s_gx + AA;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    load_tile<float, WP, HP>(s_phi, phi, x0 - 4, y0 - 2, P, false);
    load_tile<float, WA, HA>(s_p, phat, x0 - 2, y0 - 1, P, false);
    load_tile<float, WA, HA>(s_ux, ukx, x0 - 2, y0 - 1, P, true);
    load_tile<float, WA, HA>(s_uy, uky, x0 - 2, y0 - 1, P, true);
    tiles_ready();
    picard_strips_body<TX, TY, NT, VR1, VR2, WP, WA>(P, s_phi, s_p, s_ux, s_uy, s_mu, s_gx, s_gy, x0, y0,
                                                     [&](int, int, int, long long gidx, float2 &a, float2 &b) {
                                                         a = *reinterpret_cast<const float2 *>(&jx[gidx]);
                                                         b = *reinterpret_cast<const float2 *>(&jy[gidx]);
                                                     },
                                                     uox, uoy);
}

// ---------------------------------------------------------------------------
// TMA tile staging (FP32, grid width a multiple of 4 so rows are 16-byte
// aligned).  One CTA per tile: thread 0 issues one cp.async.bulk.tensor per
// input field for the tile's window, completing on an mbarrier; a window
// that crosses the domain edge (periodic wrap or wall mirror) is staged by
// the threads instead.  The wait is bounded: when it gives up, bit 0 of
// *err is set and the CTA leaves without computing.
// ---------------------------------------------------------------------------
struct TmaMaps {
    CUtensorMap m[4];
};

constexpr unsigned TMA_WAIT_POLLS = 1u << 20;   // about a second of polling at most

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *b, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(b)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *b, unsigned parity)
{
    for (unsigned i = 0; i < TMA_WAIT_POLLS; ++i)
        if (mbar_try_wait(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load_2d(float *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *b)
{
    asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(b))
                 : "memory");
}

// Shared memory of a TMA-staged tile: the mbarrier and a flag in the first
// 128 bytes, then NF field windows of BW x BH floats, each starting on a
// 128-byte boundary, then EXTRA work floats.
template <int NF, int BW, int BH, int EXTRA> struct TmaTile {
    static constexpr int FS = (BW * BH + 31) / 32 * 32;
    static constexpr size_t BYTES = 128 + sizeof(float) * (NF * FS + EXTRA) + 128;   // + base alignment

    unsigned long long *bar;
    int *flag;
    float *win;
    float *work;

    // Carve the dynamic shared memory and initialise the barrier.
    __device__ __forceinline__ explicit TmaTile(unsigned char *raw)
    {
        unsigned char *base = raw + ((128u - (smem_u32(raw) & 127u)) & 127u);
        bar = reinterpret_cast<unsigned long long *>(base);
        flag = reinterpret_cast<int *>(base + 16);
        win = reinterpret_cast<float *>(base + 128);
        work = win + NF * FS;
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
    }

    // Start staging the windows at global (gx, gy) of the NF fields: by TMA
    // (returns true) or, across the domain edge, by the threads themselves.
    __device__ __forceinline__ bool issue(const KP<float> &P, const TmaMaps &tm, const float *const *src,
                                          unsigned oddmask, int gx, int gy)
    {
        const bool inner = gx >= 0 && gy >= 0 && gx + BW <= P.nx && gy + BH <= P.ny;
        if (!inner) {
#pragma unroll
            for (int f = 0; f < NF; ++f)
                load_tile_mapped<float, BW, BH>(win + f * FS, src[f], gx, gy, P, (oddmask >> f) & 1u);
        } else if (threadIdx.x == 0) {
            mbar_expect_tx(bar, (unsigned)(NF * BW * BH * sizeof(float)));
#pragma unroll
            for (int f = 0; f < NF; ++f) tma_load_2d(win + f * FS, &tm.m[f], gx, gy, bar);
        }
        return inner;
    }

    // Make the staged windows readable by every thread; false (for the whole
    // CTA) when the TMA wait gave up, after recording it in *err and giving
    // the copies in flight a second bounded wait to land before the CTA
    // leaves (a copy that lands after that can still write this shared
    // memory: the host then refuses further steps on the handle).
    __device__ __forceinline__ bool wait(bool by_tma, unsigned *err)
    {
        if (by_tma && threadIdx.x == 0) {
            *flag = mbar_wait_bounded(bar, 0) ? 1 : 0;
            if (!*flag) {
                atomicOr(err, 1u);
                mbar_wait_bounded(bar, 0);
            }
        }
        __syncthreads();
        if (!by_tma) return true;
        const bool ok = *flag != 0;
        if (ok) mbar_try_wait(bar, 0);   // completed phase: acquires the TMA writes
        return ok;
    }

    __device__ __forceinline__ bool load(const KP<float> &P, const TmaMaps &tm, const float *const *src,
                                         unsigned oddmask, int gx, int gy, unsigned *err)
    {
        return wait(issue(P, tm, src, oddmask, gx, gy), err);
    }
};

__device__ __forceinline__ void tile_origin(int TX, int TY, int &x0, int &y0, const KP<float> &P)
{
    const int ntx = (P.nx + TX - 1) / TX;
    const int ty = (int)blockIdx.x / ntx;
    x0 = ((int)blockIdx.x - ty * ntx) * TX;
    y0 = ty * TY;
}

// Filter pass with TMA staging, one CTA per TX x TY tile: windows
// (TX + 16) x (TY + 2R) from (x0 - 8, y0 - R) of p_hat, u_hat_x, u_hat_y.
template <int TX, int TY, int R, int VR> struct FLTGeom {
    static constexpr int BW = TX + 16, BH = TY + 2 * R, NT = (TX / 2) * (TY / VR);
    using Tile = TmaTile<3, BW, BH, 0>;
};

template <int TX, int TY, int R, int VR, int MINB>
__global__ void __launch_bounds__((TX / 2) * (TY / VR), MINB)
k_filter_tma(const __grid_constant__ TmaMaps tm, KP<float> P, const float *__restrict__ pin,
             const float *__restrict__ uxin, const float *__restrict__ uyin, float *__restrict__ pout,
             float *__restrict__ uxout, float *__restrict__ uyout, unsigned *err)
{
    using G = FLTGeom<TX, TY, R, VR>;
    constexpr int BW = G::BW, FS = G::Tile::FS, RP = (R + 1) & ~1, OFF = 8 - RP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename G::Tile tile(smem_raw);
    const float *src[3] = {pin, uxin, uyin};
    int x0, y0;
    tile_origin(TX, TY, x0, y0, P);
    if (!tile.load(P, tm, src, 6u, x0 - 8, y0 - R, err)) return;
    const float *sp = tile.win + OFF;
    filter_strips_body<TX, TY, R, VR, BW>(P, sp, sp + FS, sp + 2 * FS, x0, y0, pout, uxout, uyout);
}

// RK3 stage with TMA staging, one CTA per TX x TY tile: windows
// (TX + 16) x (TY + 12) of phi^n and of the incoming increment d from
// (x0 - 8, y0 - 6).  psi = phi^n + d is formed in the phi window; mu and J
// then use a work area that begins at the consumed d window.
template <int TX, int TY> struct RKTGeom {
    using G = RKGeom<TX, TY>;
    static constexpr int BW = TX + 16, BH = TY + 12;
    static constexpr int FS = (BW * BH + 31) / 32 * 32;
    static constexpr int WORK = G::W4 * G::H4 + 2 * G::W2 * G::H2;
    static_assert(WORK >= FS && (BW * BH) % 4 == 0, "the work area covers the d window");
    using Tile = TmaTile<2, BW, BH, WORK - FS>;
};

template <int TX, int TY, int NT, int VR1, int VR2, int VR3, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_rk_tma(const __grid_constant__ TmaMaps tm, KP<float> P, const float *__restrict__ phi,
         const float *__restrict__ din, const float *__restrict__ dbar, float *__restrict__ out, float a, float b,
         int last, float *__restrict__ philo, unsigned *err)
{
    using T = RKTGeom<TX, TY>;
    using G = RKGeom<TX, TY>;
    constexpr int BW = T::BW, FS = T::FS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Tile tile(smem_raw);
    float *s_mu = tile.win + FS;
    float *s_jx = s_mu + G::W4 * G::H4;
    float *s_jy = s_jx + G::W2 * G::H2;
    const float *src[2] = {phi, din};
    int x0, y0;
    tile_origin(TX, TY, x0, y0, P);
    const bool by_tma = tile.issue(P, tm, src, 0u, x0 - 8, y0 - 6);
    // dbar of this thread's output strip (one strip per thread), requested
    // while the windows arrive
    static_assert((TX / 2) * (TY / VR3) == NT, "one output strip per thread");
    const int lx = 2 * ((int)threadIdx.x % (TX / 2)), r0 = ((int)threadIdx.x / (TX / 2)) * VR3;
    float2 pbv[VR3];   // dbar, then a dbar + b d
#pragma unroll
    for (int i = 0; i < VR3; ++i) pbv[i] = f2(0.0f);
    if (a != 0.0f) {
        const int X = x0 + lx;
#pragma unroll
        for (int i = 0; i < VR3; ++i) {
            const int Y = y0 + r0 + i;
            if (X < P.nx && Y < P.ny) pbv[i] = __ldg(reinterpret_cast<const float2 *>(&dbar[(long long)Y * P.nx + X]));
        }
    }
    if (!tile.wait(by_tma, err)) return;
    // the part of the stage's increment that needs no stencil, a dbar + b d,
    // at this thread's strip; then psi = phi^n + d over the window
    const float2 aa = f2(a), bb = f2(b);
#pragma unroll
    for (int i = 0; i < VR3; ++i) pbv[i] = fma2(aa, pbv[i], mul2(bb, lds2(tile.win + FS, (r0 + i + 6) * BW + lx + 8)));
    __syncthreads();
    for (int k = 4 * (int)threadIdx.x; k < BW * T::BH; k += 4 * NT) {
        float4 p = *reinterpret_cast<const float4 *>(tile.win + k);
        const float4 d = *reinterpret_cast<const float4 *>(tile.win + FS + k);
        p.x += d.x; p.y += d.y; p.z += d.z; p.w += d.w;
        *reinterpret_cast<float4 *>(tile.win + k) = p;
    }
    __syncthreads();
    rk_strips_body<TX, TY, NT, VR1, VR2, VR3, T::BW>(
        P, tile.win + 2, s_mu, s_jx, s_jy, x0, y0, [&](int i, long long gidx, float2 L) {
            float2 r = fma2(bb, L, pbv[i]);
            if (last) r = add_hi_lo(__ldg(reinterpret_cast<const float2 *>(&phi[gidx])), r, philo + gidx);
            *reinterpret_cast<float2 *>(&out[gidx]) = r;
        });
}

// Picard sweep with TMA staging, one CTA per TX x TY tile: windows
// (TX + 8) x (TY + 4) from (x0 - 4, y0 - 2) of phi, p_hat, u^k_x, u^k_y;
// mu and grad phi in the work area.  (j through two more windows, at the
// two CTAs per SM their shared memory leaves, measured slower than these
// global loads at three.)
template <int TX, int TY> struct PCTGeom {
    using G = PSGeom<TX, TY>;
    static constexpr int BW = TX + 8, BH = TY + 4;
    static constexpr int EXTRA = 3 * G::WA * G::HA;
    using Tile = TmaTile<4, BW, BH, EXTRA>;
};

template <int TX, int TY, int NT, int VR1, int VR2, int MINB>
__global__ void __launch_bounds__(NT, MINB)
k_picard_tma(const __grid_constant__ TmaMaps tm, KP<float> P, const float *__restrict__ phi,
             const float *__restrict__ phat, const float *__restrict__ jx, const float *__restrict__ jy,
             const float *__restrict__ ukx, const float *__restrict__ uky, float *__restrict__ uox,
             float *__restrict__ uoy, unsigned *err)
{
    using T = PCTGeom<TX, TY>;
    using G = PSGeom<TX, TY>;
    constexpr int BW = T::BW, FS = T::Tile::FS, AA = G::WA * G::HA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename T::Tile tile(smem_raw);
    float *s_mu = tile.work;
    float *s_gx = s_mu + AA;
    float *s_gy = s_gx + AA;
    const float *src[4] = {phi, phat, ukx, uky};
    int x0, y0;
    tile_origin(TX, TY, x0, y0, P);
    const bool by_tma = tile.issue(P, tm, src, 12u, x0 - 4, y0 - 2);
    // j of this thread's output strip (one strip per thread), requested while
    // the windows arrive
    static_assert((TX / 2) * (TY / VR2) == NT, "one output strip per thread");
    float2 pjx[VR2], pjy[VR2];
    {
        const int lx = 2 * ((int)threadIdx.x % (TX / 2)), r0 = ((int)threadIdx.x / (TX / 2)) * VR2;
        const int X = x0 + lx;
#pragma unroll
        for (int i = 0; i < VR2; ++i) {
            const int Y = y0 + r0 + i;
            pjx[i] = pjy[i] = f2(0.0f);
            if (X < P.nx && Y < P.ny) {
                const long long gidx = (long long)Y * P.nx + X;
                pjx[i] = __ldg(reinterpret_cast<const float2 *>(&jx[gidx]));
                pjy[i] = __ldg(reinterpret_cast<const float2 *>(&jy[gidx]));
            }
        }
    }
    if (!tile.wait(by_tma, err)) return;
    const float *st = tile.win;
    // p_hat and u^k from (x0 - 2, y0 - 1): one row and two columns into their windows
    picard_strips_body<TX, TY, NT, VR1, VR2, BW, BW>(
        P, st, st + FS + BW + 2, st + 2 * FS + BW + 2, st + 3 * FS + BW + 2, s_mu, s_gx, s_gy, x0, y0,
        [&](int i, int, int, long long, float2 &a, float2 &b) {
            a = pjx[i];
            b = pjy[i];
        },
        uox, uoy);
}

// ---------------------------------------------------------------------------
// Pass 1 for FP32 at the default relaxation rates (the FAST form of
// k_collide_stream), x periodic, nx a multiple of 4: thread (lane, warp)
// collides the node pair X = x0 - 2 + 2 lane, X + 1 of collision-region row
// Y = y0 - 1 + warp, so a warp is one 64-column row (TX = 60 interior
// columns).  Streaming splits by direction: the x part of every move is a
// warp shuffle (post-collision values are pre-shifted along x, so column x
// then holds f*_q(x - c_qx)); directions with c_qy = 0 are then pulled from
// the thread's own registers and the six with c_qy != 0 from the rows above
// and below through shared memory.  Walls in y use halfway bounce-back from
// the same arrays.  Only TX, the interior rows (TY) and the window layout
// differ from k_collide_stream; the arithmetic is paired FP32.
// ---------------------------------------------------------------------------
template <typename S> struct Codec2;
template <> struct Codec2<float> {
    static __device__ __forceinline__ float2 load(const float *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    static __device__ __forceinline__ void store(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
};
template <> struct Codec2<__nv_bfloat16> {
    static __device__ __forceinline__ float2 load(const __nv_bfloat16 *p)
    {
        return __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    }
    static __device__ __forceinline__ void store(__nv_bfloat16 *p, float2 v)
    {
        *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(v.x, v.y);
    }
};
template <> struct Codec2<__half> {   // the 2^14 scale of Codec<__half, float>
    static __device__ __forceinline__ float2 load(const __half *p)
    {
        return mul2(__half22float2(__ldg(reinterpret_cast<const __half2 *>(p))), f2(1.0f / 16384.0f));
    }
    static __device__ __forceinline__ void store(__half *p, float2 v)
    {
        *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x * 16384.0f, v.y * 16384.0f);
    }
};

// Isotropic gradient of a field at the pair centred on index i of a window
// of row stride W (rows i - W, i, i + W); c returns the centre pair.
__device__ __forceinline__ void iso_grad_pair(const float *s, int i, int W, float2 &dx, float2 &dy, float2 &c)
{
    float2 Ds, Us, Dc, Uc, Dn, Un;
    iso_row(lds2(s, i - W - 2), lds2(s, i - W), lds2(s, i - W + 2), Ds, Us);
    c = lds2(s, i);
    iso_row(lds2(s, i - 2), c, lds2(s, i + 2), Dc, Uc);
    iso_row(lds2(s, i + W - 2), lds2(s, i + W), lds2(s, i + W + 2), Dn, Un);
    dx = iso_dx(Ds, Dc, Dn);
    dy = sub2(Un, Us);
}

// kappa div T, T = (gy^2, -gx gy; -gx gy, gx^2), at the pair centred on i of
// the grad phi arrays (row stride W); gxc, gyc return grad phi at the pair.
__device__ __forceinline__ void surface_force_pair(const float *sgx, const float *sgy, int i, int W, float kappa,
                                                   float2 &Fsx, float2 &Fsy, float2 &gxc, float2 &gyc)
{
    float2 Dxx[3], Dxy[3], Uxy[3], Uyy[3], dummy;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int r = i + (k - 1) * W;
        const float2 al = lds2(sgx, r - 2), ac = lds2(sgx, r), ar = lds2(sgx, r + 2);
        const float2 bl = lds2(sgy, r - 2), bc = lds2(sgy, r), br = lds2(sgy, r + 2);
        if (k == 1) {
            gxc = ac;
            gyc = bc;
        }
        iso_row(mul2(bl, bl), mul2(bc, bc), mul2(br, br), Dxx[k], dummy);
        const float2 m1 = f2(-1.0f);
        iso_row(mul2(m1, mul2(al, bl)), mul2(m1, mul2(ac, bc)), mul2(m1, mul2(ar, br)), Dxy[k], Uxy[k]);
        iso_row(mul2(al, al), mul2(ac, ac), mul2(ar, ar), dummy, Uyy[k]);
    }
    const float2 kp = f2(kappa);
    Fsx = mul2(kp, add2(iso_dx(Dxx[0], Dxx[1], Dxx[2]), sub2(Uxy[2], Uxy[0])));
    Fsy = mul2(kp, add2(iso_dx(Dxy[0], Dxy[1], Dxy[2]), sub2(Uyy[2], Uyy[0])));
}

// Populations from moments (the inverse of the MRT matrix of Sec. III.A), paired.
__device__ __forceinline__ void from_moments2(const float2 m[9], float2 f[9])
{
    const float2 r = mul2(m[0], f2(1.0f / 9.0f)), e = mul2(m[1], f2(1.0f / 36.0f)), ep = mul2(m[2], f2(1.0f / 36.0f));
    const float2 jx = mul2(m[3], f2(1.0f / 6.0f)), qx = mul2(m[4], f2(1.0f / 12.0f));
    const float2 jy = mul2(m[5], f2(1.0f / 6.0f)), qy = mul2(m[6], f2(1.0f / 12.0f));
    const float2 pxx = mul2(m[7], f2(0.25f)), pxy = mul2(m[8], f2(0.25f));
    f[0] = fma2(f2(4.0f), sub2(ep, e), r);
    const float2 ax = fma2(f2(-2.0f), ep, sub2(r, e));
    const float2 sx = fma2(f2(-2.0f), qx, jx), sy = fma2(f2(-2.0f), qy, jy);
    const float2 axp = add2(ax, pxx), axm = sub2(ax, pxx);
    f[1] = add2(axp, sx);
    f[2] = add2(axm, sy);
    f[3] = sub2(axp, sx);
    f[4] = sub2(axm, sy);
    const float2 dg = add2(fma2(f2(2.0f), e, r), ep);
    const float2 tx = add2(jx, qx), ty = add2(jy, qy);
    const float2 tp = add2(tx, ty), tm = sub2(tx, ty);
    const float2 dgp = add2(dg, pxy), dgm = sub2(dg, pxy);
    f[5] = add2(dgp, tp);
    f[6] = sub2(dgm, tm);
    f[7] = sub2(dgp, tp);
    f[8] = add2(dgm, tm);
}

// Shift post-collision values along x by c_qx (the x part of streaming):
// afterwards the pair holds f*_q(x - c_qx), f*_q(x + 1 - c_qx).
template <int CX> __device__ __forceinline__ float2 xshift(float2 v)
{
    if constexpr (CX == 1) return make_float2(__shfl_up_sync(0xffffffffu, v.y, 1), v.x);
    else if constexpr (CX == -1) return make_float2(v.y, __shfl_down_sync(0xffffffffu, v.x, 1));
    else return v;
}

template <int TX, int TY> struct CPGeom {
    static_assert(TX == 60, "a warp covers the 64 columns x0 - 2 .. x0 + 61");
    static constexpr int NT = 32 * (TY + 2);
    static constexpr int BW = TX + 16, BH = TY + 6;   // phi, p, ux, uy windows from (x0 - 8, y0 - 3)
    static constexpr int W2 = TX + 8, H2 = TY + 4;    // mu, grad phi from (x0 - 4, y0 - 2)
    static constexpr int WH = 64, HH = TY + 2;        // shifted post-collision values, collision region
    static constexpr int EXTRA = 3 * W2 * H2 + 12 * WH * HH;
    using Tile = TmaTile<4, BW, BH, EXTRA>;
};

template <typename S, int TX, int TY, int VR1>
__global__ void __launch_bounds__(32 * (TY + 2), 2)
k_collide_pairs(const __grid_constant__ TmaMaps tm, KP<float> P, const S *__restrict__ fin,
                const S *__restrict__ gin, S *__restrict__ fout, S *__restrict__ gout,
                const float *__restrict__ phi, const float *__restrict__ pfl, const float *__restrict__ ux,
                const float *__restrict__ uy, const float *__restrict__ upx, const float *__restrict__ upy,
                const float *__restrict__ uhx, const float *__restrict__ uhy, const float *__restrict__ philo,
                float *__restrict__ dbar, float *__restrict__ phat, float *__restrict__ jxo, float *__restrict__ jyo,
                unsigned *err)
{
    using G = CPGeom<TX, TY>;
    constexpr int BW = G::BW, W2 = G::W2, H2 = G::H2, WH = G::WH, HH = G::HH, FS = G::Tile::FS;
    constexpr int A2 = W2 * H2, AH = WH * HH;
    static_assert(H2 % VR1 == 0, "strips must tile the region");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    typename G::Tile tile(smem_raw);
    const float *s_phi = tile.win;
    const float *s_p = tile.win + FS;
    const float *s_ux = tile.win + 2 * FS;
    const float *s_uy = tile.win + 3 * FS;
    float *s_mu = tile.work;
    float *s_gx = s_mu + A2;
    float *s_gy = s_gx + A2;
    float *s_h = s_gy + A2;   // [12][HH][WH]: f then g, directions 2, 4, 5, 6, 7, 8

    int x0, y0;
    tile_origin(TX, TY, x0, y0, P);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int X = x0 - 2 + 2 * lane, Y = y0 - 1 + warp;
    const bool ghost = !P.py && (Y < 0 || Y >= P.ny);

    // stage the windows, and meanwhile read this pair's populations: only the
    // moments that relax at rates other than 1 are needed from them
    const float *src[4] = {phi, pfl, ux, uy};
    const bool by_tma = tile.issue(P, tm, src, 12u, x0 - 8, y0 - 3);
    float2 m3i = f2(0.0f), m5i = f2(0.0f), m4i = f2(0.0f), m6i = f2(0.0f), m7i = f2(0.0f), m8i = f2(0.0f);
    float2 upx2 = f2(0.0f), upy2 = f2(0.0f), uhx2 = f2(0.0f), uhy2 = f2(0.0f), plo2 = f2(0.0f);
    if (!ghost) {
        int fl;
        const int gidx = map_axis(Y, P.ny, P.py, fl) * P.nx + map_axis(X, P.nx, 1, fl);
        const unsigned N32 = P.N32;
        float2 a[9], b[9];
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const unsigned o = (unsigned)gidx + (unsigned)q * N32;
            a[q] = Codec2<S>::load(fin + o);
            b[q] = Codec2<S>::load(gin + o);
        }
        plo2 = __ldg(reinterpret_cast<const float2 *>(philo + gidx));
        upx2 = __ldg(reinterpret_cast<const float2 *>(upx + gidx));
        upy2 = __ldg(reinterpret_cast<const float2 *>(upy + gidx));
        uhx2 = __ldg(reinterpret_cast<const float2 *>(uhx + gidx));
        uhy2 = __ldg(reinterpret_cast<const float2 *>(uhy + gidx));
        m3i = add2(sub2(a[1], a[3]), sub2(sub2(a[5], a[6]), sub2(a[7], a[8])));
        m5i = add2(sub2(a[2], a[4]), sub2(add2(a[5], a[6]), add2(a[7], a[8])));
        const float2 d58 = sub2(sub2(b[5], b[6]), sub2(b[7], b[8]));
        const float2 d56 = sub2(add2(b[5], b[6]), add2(b[7], b[8]));
        m4i = fma2(f2(2.0f), sub2(b[3], b[1]), d58);
        m6i = fma2(f2(2.0f), sub2(b[4], b[2]), d56);
        m7i = sub2(add2(b[1], b[3]), add2(b[2], b[4]));
        m8i = sub2(add2(b[5], b[7]), add2(b[6], b[8]));
        if constexpr (Mixed<float, S>::on) {   // the stored words leave out w_q (3 p_hat + s_q(u^{n-1})),
            // whose m4, m6, m7, m8 are -u_x, -u_y, u_x^2 - u_y^2, u_x u_y (p_hat cancels)
            m4i = sub2(m4i, upx2);
            m6i = sub2(m6i, upy2);
            m7i = add2(m7i, fma2(upx2, upx2, mul2(f2(-1.0f), mul2(upy2, upy2))));
            m8i = fma2(upx2, upy2, m8i);
        }
    }
    if (!tile.wait(by_tma, err)) return;

    {   // mu and grad phi on (x0 - 4 .. x0 + TX + 3) x (y0 - 2 .. y0 + TY + 1)
        constexpr int NP = W2 / 2, NB = H2 / VR1, NI = NP * NB;
        const float2 fb = f2(4.0f * P.beta), nk = f2(-P.kappa);
        for (int it = threadIdx.x; it < NI; it += G::NT) {
            int pr, bd;
            band_item<NP, NB>(it, pr, bd);
            const int lx = 2 * pr, r0 = bd * VR1;
            float2 C[VR1 + 2], D[VR1 + 2], Sm[VR1 + 2];
#pragma unroll
            for (int k = 0; k < VR1 + 2; ++k) {
                const int row = (r0 + k) * BW + lx + 4;   // window column of region column lx
                const float2 l = lds2(s_phi, row - 2), c = lds2(s_phi, row), r = lds2(s_phi, row + 2);
                C[k] = c;
                D[k] = make_float2(c.y - l.y, r.x - c.x);
                Sm[k] = make_float2(c.y + l.y, r.x + c.x);
            }
#pragma unroll
            for (int i = 0; i < VR1; ++i) {
                const float2 gx = iso_dx(D[i], D[i + 1], D[i + 2]);
                const float2 gy = fma2(f2(1.0f / 3.0f), sub2(C[i + 2], C[i]),
                                       mul2(f2(1.0f / 12.0f), sub2(Sm[i + 2], Sm[i])));
                const float2 lap = fma2(f2(2.0f / 3.0f), add2(Sm[i + 1], add2(C[i + 2], C[i])),
                                        fma2(f2(1.0f / 6.0f), add2(Sm[i + 2], Sm[i]),
                                             mul2(f2(-10.0f / 3.0f), C[i + 1])));
                const float2 ph = C[i + 1];
                const int o = (r0 + i) * W2 + lx;
                sts2(s_mu, o, fma2(fb, sub2(mul2(mul2(ph, ph), ph), ph), mul2(nk, lap)));
                sts2(s_gx, o, gx);
                sts2(s_gy, o, gy);
            }
        }
    }
    __syncthreads();

    // ---- forces and collision of this pair
    float2 f[9], g[9], phc = f2(0.0f);
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = g[q] = f2(0.0f);
    if (!ghost) {
        const int i2 = (warp + 1) * W2 + 2 + 2 * lane;   // region of mu, grad phi
        const int iw = (warp + 2) * BW + 6 + 2 * lane;   // windows of phi, p, u
        const float2 ph = lds2(s_phi, iw);
        phc = ph;
        float2 rho, ir, nu;
        rho_nu(P, ph.x, rho.x, ir.x, nu.x);
        rho_nu(P, ph.y, rho.y, ir.y, nu.y);
        float2 dmx, dmy, mu;
        iso_grad_pair(s_mu, i2, W2, dmx, dmy, mu);
        float2 Fsx, Fsy, gxc, gyc;
        surface_force_pair(s_gx, s_gy, i2, W2, P.kappa, Fsx, Fsy, gxc, gyc);
        float2 dpx, dpy, pc, dxux, dyux, u0, dxuy, dyuy, u1;
        iso_grad_pair(s_p, iw, BW, dpx, dpy, pc);
        iso_grad_pair(s_ux, iw, BW, dxux, dyux, u0);
        iso_grad_pair(s_uy, iw, BW, dxuy, dyuy, u1);
        const float2 dr = f2(P.drho), drm = f2(P.drho * P.M);
        const float2 grx = mul2(dr, gxc), gry = mul2(dr, gyc);
        const float2 Jx = mul2(drm, dmx), Jy = mul2(drm, dmy);
        const float2 Sxx = add2(dxux, dxux), Sxy = add2(dyux, dxuy), Syy = add2(dyuy, dyuy);
        const float2 rg = sub2(rho, f2(P.g_rho_ref)), m1 = f2(-1.0f);
        float2 Fx = fma2(rg, f2(P.gx), fma2(Jx, dxux, mul2(Jy, dyux)));
        float2 Fy = fma2(rg, f2(P.gy), fma2(Jx, dxuy, mul2(Jy, dyuy)));
        Fx = fma2(nu, fma2(Sxx, grx, mul2(Sxy, gry)), add2(Fx, fma2(mul2(m1, pc), grx, Fsx)));
        Fy = fma2(nu, fma2(Sxy, grx, mul2(Syy, gry)), add2(Fy, fma2(mul2(m1, pc), gry, Fsy)));
        const float2 ax = fma2(u0, dxux, fma2(u1, dyux, sub2(u0, upx2)));
        const float2 ay = fma2(u0, dxuy, fma2(u1, dyuy, sub2(u1, upy2)));
        const float2 u00 = mul2(u0, u0), u11 = mul2(u1, u1), u01 = mul2(u0, u1);
        const float2 u2 = add2(u00, u11), uxy = sub2(u00, u11);

        {   // CH populations: only m3, m5 relax at a rate other than 1; the
            // populations are deviations from phi e_0 (see k_collide_stream)
            const float2 s = f2(P.sf[3]), oms = f2(1.0f - P.sf[3]), hs = f2(1.0f - 0.5f * P.sf[3]);
            const float2 m3 = m3i, m5 = m5i;
            const float2 em = mul2(f2(P.eta), mu), ph3u2 = mul2(f2(3.0f), mul2(ph, u2));
            const float2 pax = mul2(ph, ax), pay = mul2(ph, ay);
            float2 m[9];
            m[0] = plo2;   // m_0 relaxes to phi_hi + phi_lo
            m[1] = fma2(f2(2.0f), em, fma2(f2(-4.0f), plo2, ph3u2));
            m[2] = fma2(f2(-3.0f), em, fma2(f2(4.0f), plo2, mul2(m1, ph3u2)));
            m[3] = fma2(oms, m3, fma2(s, mul2(ph, u0), mul2(hs, pax)));
            m[4] = mul2(mul2(m1, ph), fma2(f2(0.5f), ax, u0));
            m[5] = fma2(oms, m5, fma2(s, mul2(ph, u1), mul2(hs, pay)));
            m[6] = mul2(mul2(m1, ph), fma2(f2(0.5f), ay, u1));
            m[7] = mul2(ph, uxy);
            m[8] = mul2(ph, u01);
            from_moments2(m, f);
        }
        {   // NS populations: m4, m6, m7, m8 keep part of their non-equilibrium
            const float2 bx = fma2(Fx, ir, mul2(m1, dpx)), by = fma2(Fy, ir, mul2(m1, dpy));
            const float2 bu = fma2(bx, u0, mul2(by, u1));
            const float2 Gx = mul2(Fx, ir), Gy = mul2(Fy, ir);
            const float2 G7 = mul2(f2(2.0f), fma2(bx, u0, mul2(m1, mul2(by, u1))));
            const float2 G8 = fma2(by, u0, mul2(bx, u1));
            const float2 t3 = f2(3.0f), p3 = mul2(t3, pc), u23 = mul2(t3, u2);
            float2 s78;
            s78.x = rcp(nu.x * 3.0f + 0.5f);
            s78.y = rcp(nu.y * 3.0f + 0.5f);
            const float2 o4 = f2(1.0f - P.sg[4]), o6 = f2(1.0f - P.sg[6]), o78 = sub2(f2(1.0f), s78);
            const float2 hf = f2(0.5f);
            float2 m[9];
            m[0] = p3;
            m[1] = fma2(f2(-2.0f), p3, fma2(f2(3.0f), bu, u23));
            m[2] = sub2(p3, fma2(f2(3.0f), bu, u23));
            m[3] = fma2(hf, Gx, u0);
            m[4] = fma2(o4, add2(m4i, uhx2), fma2(mul2(hf, o4), mul2(m1, Gx), sub2(mul2(m1, u0), mul2(hf, Gx))));
            m[5] = fma2(hf, Gy, u1);
            m[6] = fma2(o6, add2(m6i, uhy2), fma2(mul2(hf, o6), mul2(m1, Gy), sub2(mul2(m1, u1), mul2(hf, Gy))));
            const float2 hxy = fma2(uhx2, uhx2, mul2(m1, mul2(uhy2, uhy2)));
            m[7] = fma2(o78, sub2(m7i, hxy), fma2(mul2(hf, o78), G7, fma2(hf, G7, uxy)));
            m[8] = fma2(o78, sub2(m8i, mul2(uhx2, uhy2)), fma2(mul2(hf, o78), G8, fma2(hf, G8, u01)));
            from_moments2(m, g);
        }
    }

    // ---- streaming: x part by shuffles (every lane takes part)
    f[1] = xshift<1>(f[1]); f[5] = xshift<1>(f[5]); f[8] = xshift<1>(f[8]);
    f[3] = xshift<-1>(f[3]); f[6] = xshift<-1>(f[6]); f[7] = xshift<-1>(f[7]);
    g[1] = xshift<1>(g[1]); g[5] = xshift<1>(g[5]); g[8] = xshift<1>(g[8]);
    g[3] = xshift<-1>(g[3]); g[6] = xshift<-1>(g[6]); g[7] = xshift<-1>(g[7]);
    {
        const int o = warp * WH + 2 * lane;
        constexpr int qv[6] = {2, 4, 5, 6, 7, 8};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            sts2(s_h + k * AH, o, f[qv[k]]);
            sts2(s_h + (6 + k) * AH, o, g[qv[k]]);
        }
    }
    __syncthreads();

    // ---- y part from the neighbouring rows; post-stream moments
    if (warp < 1 || warp > TY || lane < 1 || lane > 30) return;
    const int Xn = X, Yn = Y;
    if (Xn >= P.nx || Yn >= P.ny) return;
    const int up = (warp - 1) * WH + 2 * lane, dn = (warp + 1) * WH + 2 * lane, own = warp * WH + 2 * lane;
    // slots in s_h: 0:2 1:4 2:5 3:6 4:7 5:8
    float2 fv[9], gv[9];
    fv[0] = f[0]; fv[1] = f[1]; fv[3] = f[3];
    gv[0] = g[0]; gv[1] = g[1]; gv[3] = g[3];
    const float *hf_ = s_h, *hg_ = s_h + 6 * AH;
    fv[2] = lds2(hf_ + 0 * AH, up); fv[5] = lds2(hf_ + 2 * AH, up); fv[6] = lds2(hf_ + 3 * AH, up);
    fv[4] = lds2(hf_ + 1 * AH, dn); fv[7] = lds2(hf_ + 4 * AH, dn); fv[8] = lds2(hf_ + 5 * AH, dn);
    gv[2] = lds2(hg_ + 0 * AH, up); gv[5] = lds2(hg_ + 2 * AH, up); gv[6] = lds2(hg_ + 3 * AH, up);
    gv[4] = lds2(hg_ + 1 * AH, dn); gv[7] = lds2(hg_ + 4 * AH, dn); gv[8] = lds2(hg_ + 5 * AH, dn);
    if (!P.py && Yn == 0) {   // bottom wall: 2, 5, 6 come back as the node's own 4, 7, 8
        const float *b = s_h;
#pragma unroll
        for (int d = 0; d < 2; ++d, b += 6 * AH) {
            float2 *v = d ? gv : fv;
            v[2] = lds2(b + 1 * AH, own);
            v[5] = make_float2(b[4 * AH + own - 1], b[4 * AH + own]);       // f*_7(x) = h_7(x - 1)
            v[6] = make_float2(b[5 * AH + own + 1], b[5 * AH + own + 2]);   // f*_8(x) = h_8(x + 1)
        }
    }
    if (!P.py && Yn == P.ny - 1) {   // top wall: 4, 7, 8 come back as the node's own 2, 5, 6
        const float *b = s_h;
#pragma unroll
        for (int d = 0; d < 2; ++d, b += 6 * AH) {
            float2 *v = d ? gv : fv;
            v[4] = lds2(b + 0 * AH, own);
            v[7] = make_float2(b[2 * AH + own + 1], b[2 * AH + own + 2]);   // f*_5(x) = h_5(x + 1)
            v[8] = make_float2(b[3 * AH + own - 1], b[3 * AH + own]);       // f*_6(x) = h_6(x - 1)
        }
    }
    float2 sf = fv[0], sg = gv[0];
#pragma unroll
    for (int q = 1; q < 9; ++q) {
        sf = add2(sf, fv[q]);
        sg = add2(sg, gv[q]);
    }
    const float2 jx = add2(sub2(gv[1], gv[3]), sub2(sub2(gv[5], gv[6]), sub2(gv[7], gv[8])));
    const float2 jy = add2(sub2(gv[2], gv[4]), sub2(add2(gv[5], gv[6]), add2(gv[7], gv[8])));
    const float2 pn = mul2(sg, f2(1.0f / 3.0f));
    const int nidx = Yn * P.nx + Xn;
    const unsigned N32 = P.N32;
    if constexpr (Mixed<float, S>::on) {
#pragma unroll
        for (int q = 1; q < 9; ++q) Codec2<S>::store(fout + (unsigned)nidx + (unsigned)q * N32, fv[q]);
        // g less its equilibrium at (p_hat, u^n) of this node (see s_eq), for the
        // opposite directions q, qo with c_q.u = c: 3 p_hat - 3/2 u.u + 9/2 c^2 +- 3 c
        const int iu = (warp + 2) * BW + 6 + 2 * lane;
        const float2 un0 = lds2(s_ux, iu), un1 = lds2(s_uy, iu);
        const float2 p3 = fma2(f2(-1.5f), fma2(un0, un0, mul2(un1, un1)), mul2(f2(3.0f), pn));
        auto store_pair = [&](int q, int qo, float2 c) {
            const float2 ev = fma2(mul2(f2(4.5f), c), c, p3), od = mul2(f2(3.0f), c), w = f2(-lattice_w(q));
            Codec2<S>::store(gout + (unsigned)nidx + (unsigned)q * N32, fma2(w, add2(ev, od), gv[q]));
            Codec2<S>::store(gout + (unsigned)nidx + (unsigned)qo * N32, fma2(w, sub2(ev, od), gv[qo]));
        };
        store_pair(1, 3, un0);
        store_pair(2, 4, un1);
        store_pair(5, 7, add2(un0, un1));
        store_pair(6, 8, sub2(un1, un0));
    } else {
        Codec2<S>::store(fout + nidx, add2(phc, fv[0]));
#pragma unroll
        for (int q = 1; q < 9; ++q) Codec2<S>::store(fout + (unsigned)nidx + (unsigned)q * N32, fv[q]);
#pragma unroll
        for (int q = 0; q < 9; ++q) Codec2<S>::store(gout + (unsigned)nidx + (unsigned)q * N32, gv[q]);
    }
    sts2(dbar, nidx, sf);
    sts2(phat, nidx, pn);
    sts2(jxo, nidx, jx);
    sts2(jyo, nidx, jy);
}

// ---------------------------------------------------------------------------
// Initialisation: f = f_eq(phi, mu(phi), u) (Eq. feq_CH), g = g_eq(p, u) (Eq. geq),
// written through the moment form of the equilibria.
// ---------------------------------------------------------------------------
template <typename T, typename S>
__global__ void k_init(KP<T> P, const T *__restrict__ phi, const T *__restrict__ p,
                       const T *__restrict__ ux, const T *__restrict__ uy,
                       S *__restrict__ f, S *__restrict__ g,
                       T *__restrict__ dbar, T *__restrict__ phat)
{
    const long long N = P.N;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        const int Y = (int)(k / P.nx), X = (int)(k - (long long)Y * P.nx);
        T nbv[9];
        constexpr int cxv[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        constexpr int cyv[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            int fx, fy;
            int gx = map_axis(X + cxv[q], P.nx, P.px, fx);
            int gy = map_axis(Y + cyv[q], P.ny, P.py, fy);
            nbv[q] = phi[(long long)gy * P.nx + gx];
        }
        // order in nbv: C, E, N, W, S, NE, NW, SW, SE
        const T lap = (nbv[1] + nbv[2] + nbv[3] + nbv[4]) * T(2.0 / 3.0) +
                      (nbv[5] + nbv[6] + nbv[7] + nbv[8]) * T(1.0 / 6.0) - nbv[0] * T(10.0 / 3.0);
        const T ph = nbv[0];
        const T mu = T(4) * P.beta * (ph * ph * ph - ph) - P.kappa * lap;
        const T u0 = ux[k], u1 = uy[k], u2 = u0 * u0 + u1 * u1, pc = p[k];
        const T em = P.eta * mu;
        const T mf[9] = {ph, T(2) * em - T(4) * ph + T(3) * ph * u2, T(4) * ph - T(3) * em - T(3) * ph * u2,
                         ph * u0, -ph * u0, ph * u1, -ph * u1, ph * (u0 * u0 - u1 * u1), ph * u0 * u1};
        const T mg[9] = {T(3) * pc, T(-6) * pc + T(3) * u2, T(3) * pc - T(3) * u2, u0, -u0, u1, -u1,
                         u0 * u0 - u1 * u1, u0 * u1};
        T fv[9], gv[9];
        from_moments(mf, fv);
        from_moments(mg, gv);
        T sg = T(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) sg += gv[q];
        const T pn = sg * T(1.0 / 3.0);
        dbar[k] = T(0);   // sum f_eq = phi: the post-stream increment starts at zero
        phat[k] = pn;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            if (Mixed<T, S>::on) {
                if (q == 0) continue;
                f[q * N + k] = Codec<S, T>::store(fv[q]);
                g[q * N + k] = Codec<S, T>::store(gv[q] - T(lattice_w(q)) * (T(3) * pn + s_eq(q, u0, u1)));
            } else {
                f[q * N + k] = Codec<S, T>::store(fv[q]);
                g[q * N + k] = Codec<S, T>::store(gv[q]);
            }
        }
    }
}

// out = s * in, element-wise.
template <typename T>
__global__ void k_scale(const T *__restrict__ in, T s, T *__restrict__ out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = s * in[k];
}

// phi as a pair of floats: hi = phi rounded, lo = the rest rounded, and back.
static __global__ void k_split(const double *__restrict__ in, float *__restrict__ hi, float *__restrict__ lo, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const double x = in[k];
        const float h = (float)x;
        hi[k] = h;
        lo[k] = (float)(x - (double)h);
    }
}
static __global__ void k_join(const float *__restrict__ hi, const float *__restrict__ lo, double *__restrict__ out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = (double)hi[k] + (double)lo[k];
}

// Element-wise type conversion (host double fields <-> device arithmetic type).
template <typename A, typename B>
__global__ void k_cast(const A *__restrict__ in, B *__restrict__ out, long long n)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        out[k] = (B)in[k];
}

// ---------------------------------------------------------------------------
// Diagnostics: per-block FP64 partial sums (Sec. IV.C volume, Sec. IV.E
// centroid and rise velocity), reduced by warp shuffles; a second kernel
// folds the block partials in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int NDIAG = 11;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

constexpr int DSEG = 16;  // nodes a thread sums before adding to its sums
static_assert(DSEG % 2 == 0, "whole segments are summed as node pairs");

// A float accumulator carried as an unevaluated sum hi + lo (Knuth's TwoSum
// after every addition): a segment of FP32 terms is summed without rounding
// error beyond the order of the square of the unit roundoff, and enters the
// FP64 sums as (double)hi + (double)lo.
struct FFAcc {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = hi + x;
        lo += two_sum_err(hi, x, s);
        hi = s;
    }
    // this += b: TwoSum of the high parts, the low parts and that error
    // added, then renormalised; the error is of the order of the square of
    // the unit roundoff times |this + b|
    __device__ __forceinline__ void add(const FFAcc &b)
    {
        const float s = hi + b.hi;
        const float e = two_sum_err(hi, b.hi, s) + (lo + b.lo);
        hi = s + e;
        lo = two_sum_err(s, e, hi);
    }
    // this += b * y for an integer y exactly representable as a float
    __device__ __forceinline__ void add_scaled(const FFAcc &b, float y)
    {
        FFAcc t;
        t.hi = b.hi * y;
        t.lo = fmaf(b.hi, y, -t.hi) + b.lo * y;
        add(t);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Two FFAcc side by side in paired FP32 (one lane per node of a pair).
struct FFAcc2 {
    float2 hi = make_float2(0.0f, 0.0f), lo = make_float2(0.0f, 0.0f);
    __device__ __forceinline__ void add(float2 x)
    {
        const float2 s = add2(hi, x);
        const float2 bp = sub2(s, hi), ap = sub2(s, bp);
        lo = add2(lo, add2(sub2(hi, ap), sub2(x, bp)));   // TwoSum error, lane by lane
        hi = s;
    }
    // the two lanes' sums, as one float pair
    __device__ __forceinline__ FFAcc merged() const
    {
        FFAcc a, b;
        a.hi = hi.x;
        a.lo = lo.x;
        b.hi = hi.y;
        b.lo = lo.y;
        a.add(b);
        return a;
    }
};

template <typename T>
__global__ void __launch_bounds__(256, 2)
k_diag_partial(int nx, int ny, const T *__restrict__ phi, const T *__restrict__ p, const T *__restrict__ ux,
               const T *__restrict__ uy, double *__restrict__ part)
{
    // each thread accumulates at most DSEG nodes of a row (a segment) before
    // adding the segment to its sums.
    // FP64 handles add in FP64 throughout.  FP32 handles form every term
    // exactly as a float pair -- w = (1 - phi)/2 by TwoSum (the halving is
    // exact), w uy by an FMA for the product's error -- sum the segment in
    // FFAcc and the segments in float-pair sums, which go to FP64 once per
    // thread: the sums match FP64 sums of the same FP32 fields to the order
    // of the FP64 rounding (each segment is off by at most (15u)^2 of the sum
    // of its |terms|, u = 2^-24, each float-pair addition by about u^2).
    double s_ph = 0.0, s_v = 0.0, s_w = 0.0, s_wy = 0.0, s_wv = 0.0;
    FFAcc f_ph, f_v, f_w, f_wy, f_wv;   // FP32 handles: the segments' sums, as float pairs
    long long n_pos = 0, n_neg = 0, s_y = 0, n_bad = 0;
    T mx = T(-INFINITY), mn = T(INFINITY);
    // work items: a row cut into chunks of DSEG * blockDim.x nodes (one
    // segment per thread), dealt to the blocks in turn, so that the blocks
    // finish together
    const int chunk = DSEG * (int)blockDim.x, cpr = (nx + chunk - 1) / chunk;
    for (long long item = blockIdx.x; item < (long long)ny * cpr; item += gridDim.x) {
        const int y = (int)(item / cpr), xc = (int)(item - (long long)y * cpr) * chunk;
        const long long r = (long long)y * nx;
        int npos = 0, nneg = 0;
        // one segment of DSEG nodes per thread, its loads all issued first
        {
            const int xs = xc + (int)threadIdx.x;
            T ph[DSEG], v[DSEG], pp[DSEG], uu[DSEG];
#pragma unroll
            for (int u = 0; u < DSEG; ++u) {
                const int x = xs + u * blockDim.x;
                const bool in = x < nx;
                ph[u] = in ? phi[r + x] : T(0);
                v[u] = in ? uy[r + x] : T(0);
                pp[u] = in ? p[r + x] : T(0);
                uu[u] = in ? ux[r + x] : T(0);
            }
            if constexpr (std::is_same<T, float>::value) {
                FFAcc a_ph, a_v, a_w, a_wv;
                if (xs + (DSEG - 1) * (int)blockDim.x < nx) {
                    // a whole segment: nodes u and u + 1 as the two lanes of
                    // paired FP32, the same terms as below; the finiteness of
                    // every value is tested at once by a running sum of x - x
                    // (0 for every finite x), counted one by one only when
                    // that sum is NaN
                    FFAcc2 b_ph, b_v, b_w, b_wv;
                    float2 nan_acc = f2(0.0f);
                    const float2 one = f2(1.0f), half = f2(0.5f), m1 = f2(-1.0f);
#pragma unroll
                    for (int u = 0; u < DSEG; u += 2) {
                        const float2 P = make_float2(ph[u], ph[u + 1]), V = make_float2(v[u], v[u + 1]);
                        const float2 Q = make_float2(pp[u], pp[u + 1]), U = make_float2(uu[u], uu[u + 1]);
                        const float2 om = sub2(one, P), mP = mul2(m1, P);
                        const float2 bp = sub2(om, one), ap = sub2(om, bp);
                        const float2 w = mul2(half, om);
                        const float2 wl = mul2(half, add2(sub2(one, ap), sub2(mP, bp)));   // w + wl = (1 - phi)/2
                        const float2 wv = mul2(w, V);
                        b_ph.add(P);
                        b_w.add(w);
                        b_w.lo = add2(b_w.lo, wl);
                        b_wv.add(wv);
                        b_wv.lo = add2(b_wv.lo, add2(fma2(w, V, mul2(m1, wv)), mul2(wl, V)));
                        b_v.add(make_float2(P.x < 0.0f ? V.x : 0.0f, P.y < 0.0f ? V.y : 0.0f));
                        npos += (int)(P.x > 0.0f) + (int)(P.y > 0.0f);
                        nneg += (int)(P.x < 0.0f) + (int)(P.y < 0.0f);
                        mx = fmax(mx, fmax(P.x, P.y));
                        mn = fmin(mn, fmin(P.x, P.y));
                        nan_acc = add2(nan_acc, add2(add2(sub2(P, P), sub2(V, V)), add2(sub2(Q, Q), sub2(U, U))));
                    }
                    if (isnan(nan_acc.x) || isnan(nan_acc.y)) {
#pragma unroll
                        for (int u = 0; u < DSEG; ++u)
                            n_bad += (int)!isfinite(ph[u]) + (int)!isfinite(pp[u]) + (int)!isfinite(uu[u]) +
                                     (int)!isfinite(v[u]);
                    }
                    a_ph = b_ph.merged();
                    a_v = b_v.merged();
                    a_w = b_w.merged();
                    a_wv = b_wv.merged();
                } else {   // the last, partial segment of a row
#pragma unroll
                for (int u = 0; u < DSEG; ++u) {
                    if (xs + u * blockDim.x >= nx) break;
                    const float om = 1.0f - ph[u];
                    const float w = 0.5f * om, wl = 0.5f * two_sum_err(1.0f, -ph[u], om);   // w + wl = (1 - phi)/2
                    const float wv = w * v[u];
                    a_ph.add(ph[u]);
                    a_w.add(w);
                    a_w.lo += wl;
                    a_wv.add(wv);
                    a_wv.lo += fmaf(w, v[u], -wv) + wl * v[u];
                    if (ph[u] > 0.0f) ++npos;
                    if (ph[u] < 0.0f) {
                        ++nneg;
                        a_v.add(v[u]);
                    }
                    mx = fmax(mx, ph[u]);
                    mn = fmin(mn, ph[u]);
                    n_bad += (int)!isfinite(ph[u]) + (int)!isfinite(pp[u]) + (int)!isfinite(uu[u]) + (int)!isfinite(v[u]);
                }
                }
                // the segment into the thread's float-pair sums (FP32 arithmetic:
                // FP64 is a small fraction of the FP32 rate on this GPU)
                f_ph.add(a_ph);
                f_v.add(a_v);
                f_w.add(a_w);
                f_wy.add_scaled(a_w, (float)y);
                f_wv.add(a_wv);
            } else {
                T a_ph = T(0), a_v = T(0), a_w = T(0), a_wv = T(0);
#pragma unroll
                for (int u = 0; u < DSEG; ++u) {
                    if (xs + u * blockDim.x >= nx) break;
                    const T w = (T(1) - ph[u]) * T(0.5);
                    a_ph += ph[u];
                    a_w += w;
                    a_wv += w * v[u];
                    if (ph[u] > T(0)) ++npos;
                    if (ph[u] < T(0)) {
                        ++nneg;
                        a_v += v[u];
                    }
                    mx = fmax(mx, ph[u]);
                    mn = fmin(mn, ph[u]);
                    n_bad += (int)!isfinite(ph[u]) + (int)!isfinite(pp[u]) + (int)!isfinite(uu[u]) + (int)!isfinite(v[u]);
                }
                s_ph += (double)a_ph;
                s_v += (double)a_v;
                s_w += (double)a_w;
                s_wy += (double)y * (double)a_w;
                s_wv += (double)a_wv;
            }
        }
        n_pos += npos;
        n_neg += nneg;
        s_y += (long long)y * nneg;
    }
    if constexpr (std::is_same<T, float>::value) {
        s_ph = f_ph.value();
        s_v = f_v.value();
        s_w = f_w.value();
        s_wy = f_wy.value();
        s_wv = f_wv.value();
    }
    // a non-finite phi poisons fmax/fmin only through NaN, which fmax skips:
    // the count in slot 10 reports it
    double acc[NDIAG] = {s_ph, (double)n_pos, (double)n_neg, (double)s_y, s_v, s_w, s_wy, s_wv,
                         (double)mx, (double)mn, (double)n_bad};
    __shared__ double red[NDIAG][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NDIAG; ++k) {
        double v = k == 8 ? warp_max(acc[k]) : (k == 9 ? warp_min(acc[k]) : warp_sum(acc[k]));
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < NDIAG) {
        const int k = threadIdx.x;
        double v = red[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            v = k == 8 ? fmax(v, red[k][w]) : (k == 9 ? fmin(v, red[k][w]) : v + red[k][w]);
        part[blockIdx.x * NDIAG + k] = v;
    }
}

// Warp k reduces component k of the per-block partials.
static __global__ void __launch_bounds__(32 * NDIAG) k_diag_final(int nblocks, const double *__restrict__ part,
                                                                 double *__restrict__ out)
{
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double v = k == 8 ? -INFINITY : (k == 9 ? INFINITY : 0.0);
    for (int b = lane; b < nblocks; b += 32) {
        const double x = part[b * NDIAG + k];
        v = k == 8 ? fmax(v, x) : (k == 9 ? fmin(v, x) : v + x);
    }
    v = k == 8 ? warp_max(v) : (k == 9 ? warp_min(v) : warp_sum(v));
    if (lane == 0) out[k] = v;
}

}  // namespace lbm
