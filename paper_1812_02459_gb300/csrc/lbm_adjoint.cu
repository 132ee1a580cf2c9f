// lbm_adjoint.cu -- hand-written discrete adjoint of the lattice update.
//
// The reverse sweep works on a tape of plane operations.  To differentiate
// one step, the step is re-expressed as a sequence of whole-plane
// operations -- linear combinations, products, quotients, cubes, square
// roots, the clamp of rho(phi), periodic stencils (isotropic gradient and
// Laplacian, fourth-order differences, the selective filter, the streaming
// shifts) and scalings by the differentiable parameters kappa, beta, M and
// 1/tau_f -- each executed by a small kernel and recorded.  Each operation
// has a hand-written vector-Jacobian product; the reverse sweep applies them
// in reverse order.  Across steps, sqrt(N)-style checkpointing keeps every
// k-th state, regenerates a segment with the fused forward kernels and
// reverses it step by step.  Periodic axes, FP64 or FP32 populations; the
// reverse sweep itself always runs in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <initializer_list>
#include <string>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int MAXIN = 10;
constexpr int MAXST = 25;
constexpr int NTH = 256;

enum OpKind { OP_LIN, OP_MUL, OP_DIV, OP_POW3, OP_SQRT, OP_CLAMP1, OP_RECIP, OP_STENCIL, OP_SCALEP };
enum Param { P_KAPPA, P_BETA, P_M, P_STAU, NPARAM };

struct Stencil {
    int n = 0;
    int dx[MAXST]{}, dy[MAXST]{};
    double w[MAXST]{};
};

struct Op {
    OpKind k;
    int out;
    int nin = 0;
    int in[MAXIN]{};
    double c[MAXIN]{};
    double c0 = 0.0;
    int param = -1;
    int st = -1;
};

template <typename T> struct PP { const T *p[MAXIN]; T c[MAXIN]; };
template <typename T> struct AP { T *p[MAXIN]; T c[MAXIN]; };
template <typename T> struct KSt { int n; int dx[MAXST], dy[MAXST]; T w[MAXST]; };

int blocks_for(long long N) { return (int)std::min<long long>((N + NTH - 1) / NTH, 4096); }

#define GRID_LOOP(k, N) for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (N); \
                             k += (long long)gridDim.x * blockDim.x)

template <typename T> __global__ void kk_lin(T *out, PP<T> in, int n, T c0, long long N)
{
    GRID_LOOP(k, N) {
        T acc = c0;
        for (int i = 0; i < n; ++i) acc += in.c[i] * in.p[i][k];
        out[k] = acc;
    }
}
template <typename T> __global__ void kk_lin_vjp(AP<T> ain, int n, const T *aout, long long N)
{
    GRID_LOOP(k, N) {
        const T a = aout[k];
        for (int i = 0; i < n; ++i) ain.p[i][k] += ain.c[i] * a;
    }
}
template <typename T> __global__ void kk_binary(int kind, T *out, const T *a, const T *b, long long N)
{
    GRID_LOOP(k, N) {
        const T x = a[k];
        T r;
        switch (kind) {
        case OP_MUL: r = x * b[k]; break;
        case OP_DIV: r = x / b[k]; break;
        case OP_POW3: r = x * x * x; break;
        case OP_SQRT: r = sqrt(x); break;
        case OP_CLAMP1: r = x < T(-1) ? T(-1) : (x > T(1) ? T(1) : x); break;
        default: r = T(1) / x; break;   // OP_RECIP
        }
        out[k] = r;
    }
}
template <typename T>
__global__ void kk_binary_vjp(int kind, T *aa, T *ab, const T *a, const T *b, const T *out, const T *aout, long long N)
{
    GRID_LOOP(k, N) {
        const T g = aout[k], x = a[k];
        switch (kind) {
        case OP_MUL: aa[k] += b[k] * g; ab[k] += x * g; break;
        case OP_DIV: { const T y = b[k]; aa[k] += g / y; ab[k] -= g * x / (y * y); break; }
        case OP_POW3: aa[k] += T(3) * x * x * g; break;
        case OP_SQRT: aa[k] += g / (T(2) * out[k]); break;
        case OP_CLAMP1: if (x >= T(-1) && x <= T(1)) aa[k] += g; break;
        default: aa[k] -= g / (x * x); break;   // OP_RECIP
        }
    }
}
// out(x, y) = sum_k w_k in(x + dx_k, y + dy_k) on a periodic grid; the
// transposed stencil adds sum_k w_k aout(x - dx_k, y - dy_k).
template <typename T>
__global__ void kk_stencil(T *out, const T *in, KSt<T> S, int nx, int ny, int transpose, long long N)
{
    GRID_LOOP(k, N) {
        const int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
        T acc = T(0);
        for (int i = 0; i < S.n; ++i) {
            int xx = transpose ? x - S.dx[i] : x + S.dx[i];
            int yy = transpose ? y - S.dy[i] : y + S.dy[i];
            xx %= nx; if (xx < 0) xx += nx;
            yy %= ny; if (yy < 0) yy += ny;
            acc += S.w[i] * in[(long long)yy * nx + xx];
        }
        if (transpose) out[k] += acc;
        else out[k] = acc;
    }
}
template <typename U, typename T> __global__ void kk_cast(T *out, const U *in, long long N)
{
    GRID_LOOP(k, N) out[k] = (T)in[k];
}
template <typename T> __global__ void kk_scale(T *out, const T *in, T s, long long N)
{
    GRID_LOOP(k, N) out[k] = s * in[k];
}
template <typename T> __global__ void kk_axpy(T *out, const T *in, T s, long long N)
{
    GRID_LOOP(k, N) out[k] += s * in[k];
}
// grad[p] += sum_k in[k] * aout[k] (FP64 accumulation)
template <typename T> __global__ void kk_dot(double *acc, const T *a, const T *b, long long N)
{
    double s = 0.0;
    GRID_LOOP(k, N) s += (double)a[k] * (double)b[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[NTH / 32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NTH / 32; ++w) t += red[w];
        atomicAdd(acc, t);
    }
}

// ---------------------------------------------------------------------------
// The tape engine.
// ---------------------------------------------------------------------------
template <typename T> struct Engine {
    int nx = 0, ny = 0;
    long long N = 0;
    cudaStream_t st = nullptr;
    cudaError_t err = cudaSuccess;
    std::vector<T *> val, adj;
    std::vector<T *> pool;
    std::vector<Op> tape;
    std::vector<Stencil> stencils;
    double pval[NPARAM]{};
    double *d_pgrad = nullptr;
    int nb = 1;

    void check(cudaError_t e) { if (e != cudaSuccess && err == cudaSuccess) err = e; }

    T *take()
    {
        if (!pool.empty()) { T *p = pool.back(); pool.pop_back(); return p; }
        T *p = nullptr;
        check(cudaMalloc((void **)&p, sizeof(T) * (size_t)N));
        return p;
    }
    void reset()
    {
        for (T *p : val) if (p) pool.push_back(p);
        for (T *p : adj) if (p) pool.push_back(p);
        val.clear();
        adj.clear();
        tape.clear();
    }
    void release_all()
    {
        reset();
        for (T *p : pool) cudaFree(p);
        pool.clear();
        if (d_pgrad) cudaFree(d_pgrad);
        d_pgrad = nullptr;
    }
    int newplane()
    {
        val.push_back(take());
        adj.push_back(nullptr);
        return (int)val.size() - 1;
    }
    T *A(int id)   // adjoint plane, zeroed on first use
    {
        if (!adj[id]) {
            adj[id] = take();
            check(cudaMemsetAsync(adj[id], 0, sizeof(T) * (size_t)N, st));
        }
        return adj[id];
    }
    template <typename U> int leaf(const U *src)
    {
        int id = newplane();
        if (sizeof(U) == sizeof(T))
            check(cudaMemcpyAsync(val[id], src, sizeof(T) * (size_t)N, cudaMemcpyDeviceToDevice, st));
        else
            kk_cast<U, T><<<nb, NTH, 0, st>>>(val[id], src, N);
        return id;
    }
    int lin(std::initializer_list<std::pair<int, double>> terms, double c0 = 0.0)
    {
        Op o;
        o.k = OP_LIN;
        o.c0 = c0;
        for (auto &t : terms) { o.in[o.nin] = t.first; o.c[o.nin] = t.second; ++o.nin; }
        return emit(o);
    }
    int lin_v(const int *ids, const double *cs, int n, double c0 = 0.0)
    {
        Op o;
        o.k = OP_LIN;
        o.c0 = c0;
        for (int i = 0; i < n; ++i) if (cs[i] != 0.0) { o.in[o.nin] = ids[i]; o.c[o.nin] = cs[i]; ++o.nin; }
        return emit(o);
    }
    int unary(OpKind k, int a) { Op o; o.k = k; o.in[0] = a; o.nin = 1; return emit(o); }
    int binary(OpKind k, int a, int b) { Op o; o.k = k; o.in[0] = a; o.in[1] = b; o.nin = 2; return emit(o); }
    int mul(int a, int b) { return binary(OP_MUL, a, b); }
    int div(int a, int b) { return binary(OP_DIV, a, b); }
    int sten(int a, int s) { Op o; o.k = OP_STENCIL; o.in[0] = a; o.nin = 1; o.st = s; return emit(o); }
    int scalep(int a, int p) { Op o; o.k = OP_SCALEP; o.in[0] = a; o.nin = 1; o.param = p; return emit(o); }

    KSt<T> kst(int s) const
    {
        KSt<T> K;
        K.n = stencils[s].n;
        for (int i = 0; i < K.n; ++i) { K.dx[i] = stencils[s].dx[i]; K.dy[i] = stencils[s].dy[i]; K.w[i] = (T)stencils[s].w[i]; }
        return K;
    }

    int emit(Op o)
    {
        o.out = newplane();
        T *out = val[o.out];
        switch (o.k) {
        case OP_LIN: {
            PP<T> pp{};
            for (int i = 0; i < o.nin; ++i) { pp.p[i] = val[o.in[i]]; pp.c[i] = (T)o.c[i]; }
            kk_lin<T><<<nb, NTH, 0, st>>>(out, pp, o.nin, (T)o.c0, N);
            break;
        }
        case OP_STENCIL:
            kk_stencil<T><<<nb, NTH, 0, st>>>(out, val[o.in[0]], kst(o.st), nx, ny, 0, N);
            break;
        case OP_SCALEP:
            kk_scale<T><<<nb, NTH, 0, st>>>(out, val[o.in[0]], (T)pval[o.param], N);
            break;
        default:
            kk_binary<T><<<nb, NTH, 0, st>>>((int)o.k, out, val[o.in[0]], o.nin > 1 ? val[o.in[1]] : nullptr, N);
        }
        check(cudaGetLastError());
        tape.push_back(o);
        return o.out;
    }

    void reverse()
    {
        for (int t = (int)tape.size() - 1; t >= 0; --t) {
            const Op &o = tape[t];
            if (!adj[o.out]) continue;   // nothing flows back through this operation
            const T *g = adj[o.out];
            switch (o.k) {
            case OP_LIN: {
                AP<T> ap{};
                for (int i = 0; i < o.nin; ++i) { ap.p[i] = A(o.in[i]); ap.c[i] = (T)o.c[i]; }
                kk_lin_vjp<T><<<nb, NTH, 0, st>>>(ap, o.nin, g, N);
                break;
            }
            case OP_STENCIL:
                kk_stencil<T><<<nb, NTH, 0, st>>>(A(o.in[0]), g, kst(o.st), nx, ny, 1, N);
                break;
            case OP_SCALEP:
                kk_axpy<T><<<nb, NTH, 0, st>>>(A(o.in[0]), g, (T)pval[o.param], N);
                kk_dot<T><<<std::min(nb, 1024), NTH, 0, st>>>(d_pgrad + o.param, val[o.in[0]], g, N);
                break;
            default: {
                T *aa = A(o.in[0]);
                T *ab = o.nin > 1 ? A(o.in[1]) : nullptr;
                kk_binary_vjp<T><<<nb, NTH, 0, st>>>((int)o.k, aa, ab, val[o.in[0]],
                                                     o.nin > 1 ? val[o.in[1]] : nullptr, val[o.out], g, N);
            }
            }
            check(cudaGetLastError());
        }
    }
    void seed(int id, const T *src)   // adj[id] += src
    {
        kk_axpy<T><<<nb, NTH, 0, st>>>(A(id), src, T(1), N);
        check(cudaGetLastError());
    }
};

// Stencil table indices.
enum { S_GX, S_GY, S_LAP, S_D1X, S_D1Y, S_D2X, S_D2Y, S_FILTER, S_SHIFT0 };
const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
const double WQ[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
// rows of the moment matrix (Sec. III.A Eq. D2Q9MRT) and their squared norms
const double MR[9][9] = {{1, 1, 1, 1, 1, 1, 1, 1, 1},     {-4, -1, -1, -1, -1, 2, 2, 2, 2},
                         {4, -2, -2, -2, -2, 1, 1, 1, 1},   {0, 1, 0, -1, 0, 1, -1, -1, 1},
                         {0, -2, 0, 2, 0, 1, -1, -1, 1},    {0, 0, 1, 0, -1, 1, 1, -1, -1},
                         {0, 0, -2, 0, 2, 1, 1, -1, -1},    {0, 1, -1, 1, -1, 0, 0, 0, 0},
                         {0, 0, 0, 0, 0, 1, -1, 1, -1}};
const double MN[9] = {9, 36, 36, 6, 12, 6, 12, 4, 4};

void filter_coeffs(int order, double d[6])
{
    for (int k = 0; k < 6; ++k) d[k] = 0.0;
    if (order == 5) { d[0] = 6.0 / 16; d[1] = -4.0 / 16; d[2] = 1.0 / 16; }
    else if (order == 7) { d[0] = 5.0 / 16; d[1] = -15.0 / 64; d[2] = 3.0 / 32; d[3] = -1.0 / 64; }
    else if (order == 9) {
        d[0] = 0.243527493120; d[1] = -0.204788880640; d[2] = 0.120007591680;
        d[3] = -0.045211119360; d[4] = 0.008228661760;
    } else if (order == 11) {
        d[0] = 0.215044884112; d[1] = -0.187772883589; d[2] = 0.123755948787;
        d[3] = -0.059227575576; d[4] = 0.018721609157; d[5] = -0.002999540835;
    }
}

std::vector<Stencil> make_stencils(const lbm_params &p)
{
    std::vector<Stencil> S(S_SHIFT0 + 9);
    auto add = [](Stencil &s, int dx, int dy, double w) { s.dx[s.n] = dx; s.dy[s.n] = dy; s.w[s.n] = w; ++s.n; };
    for (int q = 1; q < 9; ++q) {   // isotropic stencils, Sec. III.B Eq. (dicretized)
        if (CX[q]) add(S[S_GX], CX[q], CY[q], 3.0 * WQ[q] * CX[q]);
        if (CY[q]) add(S[S_GY], CX[q], CY[q], 3.0 * WQ[q] * CY[q]);
        add(S[S_LAP], CX[q], CY[q], 6.0 * WQ[q]);
    }
    add(S[S_LAP], 0, 0, -6.0 * (1.0 - WQ[0]));
    const int o4[4] = {-2, -1, 1, 2};
    const double w1[4] = {1.0 / 12, -8.0 / 12, 8.0 / 12, -1.0 / 12};   // Eq. (fourOrder_FDM)
    const double w2[4] = {-1.0 / 12, 16.0 / 12, 16.0 / 12, -1.0 / 12};
    for (int i = 0; i < 4; ++i) {
        add(S[S_D1X], o4[i], 0, w1[i]);
        add(S[S_D1Y], 0, o4[i], w1[i]);
        add(S[S_D2X], o4[i], 0, w2[i]);
        add(S[S_D2Y], 0, o4[i], w2[i]);
    }
    add(S[S_D2X], 0, 0, -30.0 / 12);
    add(S[S_D2Y], 0, 0, -30.0 / 12);
    double d[6];
    filter_coeffs(p.filter_order, d);
    const double a = p.filter_order ? p.filter_a : 0.0;
    add(S[S_FILTER], 0, 0, 1.0 - a * 2.0 * d[0]);   // Eq. (filter)
    for (int m = 1; m <= p.filter_order / 2; ++m) {
        add(S[S_FILTER], m, 0, -a * d[m]);
        add(S[S_FILTER], -m, 0, -a * d[m]);
        add(S[S_FILTER], 0, m, -a * d[m]);
        add(S[S_FILTER], 0, -m, -a * d[m]);
    }
    for (int q = 0; q < 9; ++q) add(S[S_SHIFT0 + q], -CX[q], -CY[q], 1.0);   // f_q(x) = f*_q(x - c_q)
    return S;
}

// Plane ids of one full state.
struct StateIds {
    int f[9], g[9], phi, p, ux, uy, uhx, uhy, upx, upy;
};
constexpr int NSTATE = 26;
int *slot(StateIds &s, int i)
{
    if (i < 9) return &s.f[i];
    if (i < 18) return &s.g[i - 9];
    int *r[8] = {&s.phi, &s.p, &s.ux, &s.uy, &s.uhx, &s.uhy, &s.upx, &s.upy};
    return r[i - 18];
}

template <typename T> struct Recorder {
    Engine<T> &E;
    const lbm_params &P;
    Recorder(Engine<T> &e, const lbm_params &p) : E(e), P(p) {}

    int gx(int a) { return E.sten(a, S_GX); }
    int gy(int a) { return E.sten(a, S_GY); }

    struct Fields { int rho, ir, nu, mu, grx, gry, Jx, Jy, Fsx, Fsy, gpx, gpy; };

    // rho, nu (Eqs. rho, dynamic_vis), mu (Eq. chemical), grad rho, J, F_s
    // (Eq. surfaceforce), grad p -- the part of the force independent of u
    Fields fields(int phi, int p)
    {
        Fields F;
        const double dr = (P.rho_H - P.rho_L) / 2.0;
        const double muH = P.rho_H * P.nu_H, muL = P.rho_L * P.nu_L;
        int c = E.unary(OP_CLAMP1, phi);
        F.rho = E.lin({{c, dr}}, (P.rho_H + P.rho_L) / 2.0);
        int mud = E.lin({{c, (muH - muL) / 2.0}}, (muH + muL) / 2.0);
        F.ir = E.unary(OP_RECIP, F.rho);
        F.nu = E.mul(mud, F.ir);
        F.mu = chem_iso(phi);
        int gphx = gx(phi), gphy = gy(phi);
        int gx2 = E.mul(gphx, gphx), gy2 = E.mul(gphy, gphy), gxy = E.mul(gphx, gphy);
        // F_s = kappa div(|grad phi|^2 I - grad phi grad phi)
        F.Fsx = E.scalep(E.lin({{gx(gy2), 1.0}, {gy(gxy), -1.0}}), P_KAPPA);
        F.Fsy = E.scalep(E.lin({{gx(gxy), -1.0}, {gy(gx2), 1.0}}), P_KAPPA);
        F.Jx = E.scalep(E.lin({{gx(F.mu), dr}}), P_M);
        F.Jy = E.scalep(E.lin({{gy(F.mu), dr}}), P_M);
        F.grx = E.lin({{gphx, dr}});
        F.gry = E.lin({{gphy, dr}});
        F.gpx = gx(p);
        F.gpy = gy(p);
        return F;
    }
    int chem_iso(int phi)   // 4 beta (phi^3 - phi) - kappa lap phi
    {
        int t = E.lin({{E.unary(OP_POW3, phi), 1.0}, {phi, -1.0}});
        return E.lin({{E.scalep(t, P_BETA), 4.0}, {E.scalep(E.sten(phi, S_LAP), P_KAPPA), -1.0}});
    }
    // F = F_p + F_s + F_nu + F_m + F_g (Sec. II.B Eq. reformNS)
    void force(const Fields &F, int p, int ux, int uy, int &Fx, int &Fy, int du[4])
    {
        du[0] = gx(ux); du[1] = gy(ux); du[2] = gx(uy); du[3] = gy(uy);
        int Sxx = E.lin({{du[0], 2.0}}), Sxy = E.lin({{du[1], 1.0}, {du[2], 1.0}}), Syy = E.lin({{du[3], 2.0}});
        int nvx = E.mul(F.nu, E.lin({{E.mul(Sxx, F.grx), 1.0}, {E.mul(Sxy, F.gry), 1.0}}));
        int nvy = E.mul(F.nu, E.lin({{E.mul(Sxy, F.grx), 1.0}, {E.mul(Syy, F.gry), 1.0}}));
        Fx = E.lin({{E.mul(p, F.grx), -1.0}, {F.Fsx, 1.0}, {nvx, 1.0}, {E.mul(F.Jx, du[0]), 1.0},
                    {E.mul(F.Jy, du[1]), 1.0}, {F.rho, P.gx}}, -P.g_rho_ref * P.gx);
        Fy = E.lin({{E.mul(p, F.gry), -1.0}, {F.Fsy, 1.0}, {nvy, 1.0}, {E.mul(F.Jx, du[2]), 1.0},
                    {E.mul(F.Jy, du[3]), 1.0}, {F.rho, P.gy}}, -P.g_rho_ref * P.gy);
    }
    void moments(const int *pop, int *m)
    {
        for (int k = 0; k < 9; ++k) m[k] = E.lin_v(pop, MR[k], 9);
    }
    void unmoments(const int *m, int *pop)
    {
        for (int q = 0; q < 9; ++q) {
            double c[9];
            for (int k = 0; k < 9; ++k) c[k] = MR[k][q] / MN[k];
            pop[q] = E.lin_v(m, c, 9);
        }
    }
    // equilibrium moments of Eq. (feq_CH) and Eq. (geq)
    void meq_ch(int phi, int mu, int ux, int uy, int *m)
    {
        int u2 = E.lin({{E.mul(ux, ux), 1.0}, {E.mul(uy, uy), 1.0}});
        int pu2 = E.mul(phi, u2);
        m[0] = E.lin({{phi, 1.0}});
        m[1] = E.lin({{mu, 2.0 * P.eta}, {phi, -4.0}, {pu2, 3.0}});
        m[2] = E.lin({{phi, 4.0}, {mu, -3.0 * P.eta}, {pu2, -3.0}});
        m[3] = E.mul(phi, ux); m[4] = E.lin({{m[3], -1.0}});
        m[5] = E.mul(phi, uy); m[6] = E.lin({{m[5], -1.0}});
        m[7] = E.mul(phi, E.lin({{E.mul(ux, ux), 1.0}, {E.mul(uy, uy), -1.0}}));
        m[8] = E.mul(phi, E.mul(ux, uy));
    }
    void meq_ns(int p, int ux, int uy, int *m)
    {
        int uxx = E.mul(ux, ux), uyy = E.mul(uy, uy);
        m[0] = E.lin({{p, 3.0}});
        m[1] = E.lin({{p, -6.0}, {uxx, 3.0}, {uyy, 3.0}});
        m[2] = E.lin({{p, 3.0}, {uxx, -3.0}, {uyy, -3.0}});
        m[3] = E.lin({{ux, 1.0}}); m[4] = E.lin({{ux, -1.0}});
        m[5] = E.lin({{uy, 1.0}}); m[6] = E.lin({{uy, -1.0}});
        m[7] = E.lin({{uxx, 1.0}, {uyy, -1.0}});
        m[8] = E.mul(ux, uy);
    }
    // L(psi) = div(lambda J_phi + q), Sec. II.A Eq. (step2), Eq. (fourOrder_FDM)
    int fd_rhs(int psi)
    {
        int g1 = E.sten(psi, S_D1X), g2 = E.sten(psi, S_D1Y);
        int lap = E.lin({{E.sten(psi, S_D2X), 1.0}, {E.sten(psi, S_D2Y), 1.0}});
        int t = E.lin({{E.unary(OP_POW3, psi), 1.0}, {psi, -1.0}});
        int mu = E.lin({{E.scalep(t, P_BETA), 4.0}, {E.scalep(lap, P_KAPPA), -1.0}});
        int m2 = E.lin({{E.mul(g1, g1), 1.0}, {E.mul(g2, g2), 1.0}}, P.grad_eps * P.grad_eps);
        int mag = E.unary(OP_SQRT, m2);
        int nxp = E.div(g1, mag), nyp = E.div(g2, mag);
        int jphi = E.lin({{mag, 1.0}, {E.mul(psi, psi), 2.0 / P.W}}, -2.0 / P.W);
        int jx = E.lin({{E.mul(jphi, nxp), P.lambda}});
        int jy = E.lin({{E.mul(jphi, nyp), P.lambda}});
        if (P.flux_correction) {
            int dmn = E.lin({{E.mul(E.sten(mu, S_D1X), nxp), 1.0}, {E.mul(E.sten(mu, S_D1Y), nyp), 1.0}});
            int qn = E.scalep(dmn, P_M);
            jx = E.lin({{jx, 1.0}, {E.mul(qn, nxp), -1.0}});
            jy = E.lin({{jy, 1.0}, {E.mul(qn, nyp), -1.0}});
        }
        return E.lin({{E.sten(jx, S_D1X), 1.0}, {E.sten(jy, S_D1Y), 1.0}});
    }

    StateIds step(StateIds s)
    {
        StateIds o;
        Fields F = fields(s.phi, s.p);
        int Fx, Fy, du[4];
        force(F, s.p, s.ux, s.uy, Fx, Fy, du);
        int ax = E.lin({{s.ux, 1.0}, {s.upx, -1.0}, {E.mul(s.ux, du[0]), 1.0}, {E.mul(s.uy, du[1]), 1.0}});
        int ay = E.lin({{s.uy, 1.0}, {s.upy, -1.0}, {E.mul(s.ux, du[2]), 1.0}, {E.mul(s.uy, du[3]), 1.0}});
        // CH collision in moment space, Eqs. (distribution_CH), (collison)
        int m[9], me[9], ms[9], fs[9];
        moments(s.f, m);
        meq_ch(s.phi, F.mu, s.ux, s.uy, me);
        int mF3 = E.mul(s.phi, ax), mF5 = E.mul(s.phi, ay);
        int mF[9] = {-1, -1, -1, mF3, E.lin({{mF3, -1.0}}), mF5, E.lin({{mF5, -1.0}}), -1, -1};
        for (int k = 0; k < 9; ++k) {
            if (k == 3 || k == 5) {   // s = 1/tau_f
                int dif = E.lin({{me[k], 1.0}, {m[k], -1.0}, {mF[k], -0.5}});
                ms[k] = E.lin({{m[k], 1.0}, {mF[k], 1.0}, {E.scalep(dif, P_STAU), 1.0}});
            } else {
                const double sk = P.s_f[k];
                if (mF[k] >= 0) ms[k] = E.lin({{m[k], 1.0 - sk}, {me[k], sk}, {mF[k], 1.0 - 0.5 * sk}});
                else ms[k] = E.lin({{m[k], 1.0 - sk}, {me[k], sk}});
            }
        }
        unmoments(ms, fs);
        // NS collision with the filtered equilibrium, Eq. (distribution_NS)
        int mg[9], mef[9], meh[9], mG[9], mgs[9], gs[9];
        moments(s.g, mg);
        int pho = E.lin({{mg[0], 1.0 / 3.0}});
        meq_ns(s.p, s.ux, s.uy, mef);
        meq_ns(pho, s.uhx, s.uhy, meh);
        int bx = E.lin({{E.mul(Fx, F.ir), 1.0}, {F.gpx, -1.0}});
        int by = E.lin({{E.mul(Fy, F.ir), 1.0}, {F.gpy, -1.0}});
        int bu = E.lin({{E.mul(bx, s.ux), 1.0}, {E.mul(by, s.uy), 1.0}});
        int fxr = E.mul(Fx, F.ir), fyr = E.mul(Fy, F.ir);
        mG[0] = -1;
        mG[1] = E.lin({{bu, 6.0}}); mG[2] = E.lin({{bu, -6.0}});
        mG[3] = fxr; mG[4] = E.lin({{fxr, -1.0}});
        mG[5] = fyr; mG[6] = E.lin({{fyr, -1.0}});
        mG[7] = E.lin({{E.mul(bx, s.ux), 2.0}, {E.mul(by, s.uy), -2.0}});
        mG[8] = E.lin({{E.mul(by, s.ux), 1.0}, {E.mul(bx, s.uy), 1.0}});
        int s78 = E.unary(OP_RECIP, E.lin({{F.nu, 3.0}}, 0.5));
        for (int k = 0; k < 9; ++k) {
            int d = E.lin({{mg[k], 1.0}, {meh[k], -1.0}});
            if (k < 7) {
                const double sk = P.s_g[k];
                if (mG[k] >= 0) mgs[k] = E.lin({{mef[k], 1.0}, {d, 1.0 - sk}, {mG[k], 1.0 - 0.5 * sk}});
                else mgs[k] = E.lin({{mef[k], 1.0}, {d, 1.0 - sk}});
            } else {
                int rel = E.mul(s78, E.lin({{d, 1.0}, {mG[k], 0.5}}));
                mgs[k] = E.lin({{mef[k], 1.0}, {d, 1.0}, {mG[k], 1.0}, {rel, -1.0}});
            }
        }
        unmoments(mgs, gs);
        // streaming and post-stream moments
        for (int q = 0; q < 9; ++q) {
            o.f[q] = E.sten(fs[q], S_SHIFT0 + q);
            o.g[q] = E.sten(gs[q], S_SHIFT0 + q);
        }
        double one[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1}, third[9], cxd[9], cyd[9];
        for (int q = 0; q < 9; ++q) { third[q] = 1.0 / 3.0; cxd[q] = CX[q]; cyd[q] = CY[q]; }
        int phibar = E.lin_v(o.f, one, 9);
        int phat = E.lin_v(o.g, third, 9);
        int jx = E.lin_v(o.g, cxd, 9), jy = E.lin_v(o.g, cyd, 9);
        // TVD-RK3, Eq. (TVD-3order)
        int p1 = E.lin({{phibar, 1.0}, {fd_rhs(phibar), 1.0}});
        int p2 = E.lin({{phibar, 0.75}, {p1, 0.25}, {fd_rhs(p1), 0.25}});
        o.phi = E.lin({{phibar, 1.0 / 3.0}, {p2, 2.0 / 3.0}, {fd_rhs(p2), 2.0 / 3.0}});
        // implicit velocity, Eq. (u), Picard sweeps
        Fields Fn = fields(o.phi, phat);
        int hir = E.lin({{Fn.ir, 0.5}});
        int ukx = s.ux, uky = s.uy;
        for (int it = 0; it < std::max(1, P.picard_iters); ++it) {
            int fx, fy, d4[4];
            force(Fn, phat, ukx, uky, fx, fy, d4);
            int nxk = E.lin({{jx, 1.0}, {E.mul(fx, hir), 1.0}});
            int nyk = E.lin({{jy, 1.0}, {E.mul(fy, hir), 1.0}});
            ukx = nxk;
            uky = nyk;
        }
        // selective filter, Eq. (filter)
        o.p = E.sten(phat, S_FILTER);
        o.ux = E.sten(ukx, S_FILTER);
        o.uy = E.sten(uky, S_FILTER);
        o.uhx = ukx; o.uhy = uky;
        o.upx = s.ux; o.upy = s.uy;
        return o;
    }

    // initial populations f = f_eq(phi0, mu(phi0), u0), g = g_eq(p0, u0)
    StateIds init(int phi0, int p0, int ux0, int uy0)
    {
        StateIds o;
        int mu = chem_iso(phi0);
        int mf[9], mg[9];
        meq_ch(phi0, mu, ux0, uy0, mf);
        meq_ns(p0, ux0, uy0, mg);
        unmoments(mf, o.f);
        unmoments(mg, o.g);
        o.phi = phi0; o.p = p0; o.ux = ux0; o.uy = uy0;
        o.uhx = ux0; o.uhy = uy0; o.upx = ux0; o.upy = uy0;
        return o;
    }
};

}  // namespace

// ---------------------------------------------------------------------------
// Reverse-mode state kept in the handle between begin and end.
// ---------------------------------------------------------------------------
struct lbm_adjoint {
    int nsteps = 0, every = 1;
    size_t planeb = 0;
    std::vector<void *> ckpt;      // checkpoints: NSTATE planes each
    std::vector<void *> seg;       // one segment of states
    void *init4 = nullptr;         // phi0, p0, ux0, uy0
    void *final_state = nullptr;   // state after nsteps
    void *lam = nullptr;           // adjoint state, NSTATE planes
    void *eng = nullptr;           // Engine<T>
    bool ready = false;
};

namespace {

lbm_status afail(lbm_handle *h, lbm_status st, const std::string &m)
{
    h->err = m;
    return st;
}

// Device pointer of state slot i (0..25) of the handle's current state.
void *state_ptr(lbm_handle *h, int i)
{
    const size_t pb = h->elem * (size_t)h->N;
    if (i < 9) return (char *)h->f[h->cur] + i * pb;
    if (i < 18) return (char *)h->g[h->cur] + (i - 9) * pb;
    void *r[8] = {h->phi, h->pf, h->ux[h->ucur], h->uy[h->ucur], h->uhx, h->uhy, h->ux[1 - h->ucur], h->uy[1 - h->ucur]};
    return r[i - 18];
}

cudaError_t copy_state_out(lbm_handle *h, void *dst)
{
    const size_t pb = h->elem * (size_t)h->N;
    for (int i = 0; i < NSTATE; ++i) {
        cudaError_t e = cudaMemcpyAsync((char *)dst + i * pb, state_ptr(h, i), pb, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
cudaError_t copy_state_in(lbm_handle *h, const void *src)
{
    const size_t pb = h->elem * (size_t)h->N;
    for (int i = 0; i < NSTATE; ++i) {
        cudaError_t e = cudaMemcpyAsync(state_ptr(h, i), (const char *)src + i * pb, pb, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The reverse sweep runs in FP64 whatever the handle's precision: the states
// regenerated by the forward kernels (type T) enter the tape converted to
// double, and the adjoint state is kept in double.
template <typename T> lbm_status run_reverse(lbm_handle *h, const double *seed, double *dphi0, double *dsigma, double *dM)
{
    using D = double;
    lbm_adjoint *A = h->adj;
    const size_t n = (size_t)h->N, pb = sizeof(T) * n, pd = sizeof(D) * n;
    Engine<D> *E = (Engine<D> *)A->eng;
    if (!E) {
        E = new Engine<D>();
        A->eng = E;
    }
    E->nx = h->grid.nx; E->ny = h->grid.ny; E->N = h->N; E->st = h->stream; E->nb = blocks_for(h->N);
    E->err = cudaSuccess;
    E->stencils = make_stencils(h->prm);
    const lbm_params &P = h->prm;
    E->pval[P_KAPPA] = 3.0 * P.sigma * P.W / 8.0;
    E->pval[P_BETA] = 3.0 * P.sigma / (4.0 * P.W);
    E->pval[P_M] = P.M;
    const double stau = 1.0 / (0.5 + P.M / (P.eta / 3.0));
    E->pval[P_STAU] = stau;
    if (!E->d_pgrad && cudaMalloc((void **)&E->d_pgrad, sizeof(double) * NPARAM) != cudaSuccess)
        return afail(h, LBM_ERR_OOM, "adjoint: parameter gradient buffer");
    cudaMemsetAsync(E->d_pgrad, 0, sizeof(double) * NPARAM, h->stream);

    // seed: dL/dphi at the final step, every other component zero
    D *lam = (D *)A->lam;
    cudaMemsetAsync(lam, 0, pd * NSTATE, h->stream);
    cudaMemcpyAsync(lam + 18 * n, seed, pd, cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    Recorder<D> R(*E, P);
    const int nseg = (A->nsteps + A->every - 1) / A->every;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int c0 = sgi * A->every, len = std::min(A->every, A->nsteps - c0);
        // regenerate the segment's states with the fused forward kernels
        if (copy_state_in(h, A->ckpt[sgi]) != cudaSuccess) return afail(h, LBM_ERR_CUDA, "adjoint: restore");
        for (int j = 0; j < len; ++j) {
            if (copy_state_out(h, (char *)A->seg[0] + (size_t)j * NSTATE * pb) != cudaSuccess)
                return afail(h, LBM_ERR_CUDA, "adjoint: segment store");
            if (j + 1 < len) {
                lbm_status st = lbm_internal_step(h);
                if (st) return st;
            }
        }
        for (int j = len - 1; j >= 0; --j) {
            E->reset();
            const T *sj = (const T *)((char *)A->seg[0] + (size_t)j * NSTATE * pb);
            StateIds in;
            for (int i = 0; i < NSTATE; ++i) *slot(in, i) = E->leaf(sj + i * n);
            StateIds out = R.step(in);
            for (int i = 0; i < NSTATE; ++i) E->seed(*slot(out, i), lam + i * n);
            E->reverse();
            for (int i = 0; i < NSTATE; ++i) {
                int id = *slot(in, i);
                if (E->adj[id]) cudaMemcpyAsync(lam + i * n, E->adj[id], pd, cudaMemcpyDeviceToDevice, h->stream);
                else cudaMemsetAsync(lam + i * n, 0, pd, h->stream);
            }
            if (E->err != cudaSuccess) return afail(h, LBM_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(E->err));
        }
    }
    // through the initialisation from (phi0, p0, u0)
    E->reset();
    const T *i4 = (const T *)A->init4;
    int phi0 = E->leaf(i4), p0 = E->leaf(i4 + n), ux0 = E->leaf(i4 + 2 * n), uy0 = E->leaf(i4 + 3 * n);
    StateIds s0 = R.init(phi0, p0, ux0, uy0);
    for (int i = 0; i < NSTATE; ++i) E->seed(*slot(s0, i), lam + i * n);
    E->reverse();
    std::vector<D> g(n, D(0));
    if (E->adj[phi0]) cudaMemcpyAsync(g.data(), E->adj[phi0], pd, cudaMemcpyDeviceToHost, h->stream);
    double pg[NPARAM];
    cudaMemcpyAsync(pg, E->d_pgrad, sizeof(pg), cudaMemcpyDeviceToHost, h->stream);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess || E->err != cudaSuccess)
        return afail(h, LBM_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e != cudaSuccess ? e : E->err));
    if (dphi0) for (size_t k = 0; k < n; ++k) dphi0[k] = (double)g[k];
    // chain to sigma and M: kappa = 3 sigma W/8, beta = 3 sigma/(4W), 1/tau_f = 1/(1/2 + 3M/eta)
    if (dsigma) *dsigma = pg[P_KAPPA] * 3.0 * P.W / 8.0 + pg[P_BETA] * 3.0 / (4.0 * P.W);
    if (dM) *dM = pg[P_M] - pg[P_STAU] * stau * stau * 3.0 / P.eta;
    E->reset();
    // leave the handle at the final state
    if (copy_state_in(h, A->final_state) != cudaSuccess) return afail(h, LBM_ERR_CUDA, "adjoint: final state");
    return LBM_OK;
}

}  // namespace

void lbm_internal_adjoint_free(lbm_handle *h)
{
    lbm_adjoint *A = h ? h->adj : nullptr;
    if (!A) return;
    for (void *p : A->ckpt) cudaFree(p);
    for (void *p : A->seg) cudaFree(p);
    cudaFree(A->init4);
    cudaFree(A->final_state);
    cudaFree(A->lam);
    if (A->eng) {
        auto *E = (Engine<double> *)A->eng;
        E->release_all();
        delete E;
    }
    delete A;
    h->adj = nullptr;
}

extern "C" {

lbm_status lbm_adjoint_begin(lbm_handle *h, int nsteps, int checkpoint_every)
{
    if (!h) return LBM_ERR_ARG;
    if (nsteps < 1 || checkpoint_every < 1) return afail(h, LBM_ERR_ARG, "nsteps and checkpoint_every must be >= 1");
    if (!h->grid.periodic_x || !h->grid.periodic_y) return afail(h, LBM_ERR_ARG, "the adjoint needs periodic axes");
    if (h->grid.precision != LBM_FP64 && h->grid.precision != LBM_FP32)
        return afail(h, LBM_ERR_ARG, "the adjoint needs FP64 or FP32 populations");
    if (!h->fresh_init) return afail(h, LBM_ERR_STATE, "lbm_adjoint_begin needs a state freshly set from fields");
    lbm_internal_adjoint_free(h);
    lbm_adjoint *A = new lbm_adjoint();
    h->adj = A;
    A->nsteps = nsteps;
    A->every = checkpoint_every;
    const size_t pb = h->elem * (size_t)h->N, sb = pb * NSTATE;
    const int nseg = (nsteps + checkpoint_every - 1) / checkpoint_every;
    auto alloc = [&](void **p, size_t b) { return cudaMalloc(p, b) == cudaSuccess; };
    bool ok = alloc(&A->init4, 4 * pb) && alloc(&A->final_state, sb) &&
              alloc(&A->lam, sizeof(double) * (size_t)h->N * NSTATE);
    A->ckpt.assign(nseg, nullptr);
    for (int i = 0; ok && i < nseg; ++i) ok = alloc(&A->ckpt[i], sb);
    A->seg.assign(1, nullptr);
    ok = ok && alloc(&A->seg[0], sb * (size_t)checkpoint_every);
    if (!ok) {
        cudaGetLastError();
        lbm_internal_adjoint_free(h);
        return afail(h, LBM_ERR_OOM, "adjoint: checkpoint allocation");
    }
    // the initial fields: phi0, p0, u0 of the fresh state
    cudaMemcpyAsync(A->init4, h->phi, pb, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync((char *)A->init4 + pb, h->pf, pb, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync((char *)A->init4 + 2 * pb, h->ux[h->ucur], pb, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync((char *)A->init4 + 3 * pb, h->uy[h->ucur], pb, cudaMemcpyDeviceToDevice, h->stream);
    for (int t = 0; t < nsteps; ++t) {
        if (t % checkpoint_every == 0 && copy_state_out(h, A->ckpt[t / checkpoint_every]) != cudaSuccess)
            return afail(h, LBM_ERR_CUDA, "adjoint: checkpoint copy");
        lbm_status st = lbm_internal_step(h);
        if (st) return st;
    }
    if (copy_state_out(h, A->final_state) != cudaSuccess) return afail(h, LBM_ERR_CUDA, "adjoint: final copy");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return afail(h, LBM_ERR_CUDA, std::string("adjoint forward: ") + cudaGetErrorString(e));
    A->ready = true;
    return LBM_OK;
}

lbm_status lbm_adjoint_end(lbm_handle *h, const double *dL_dphi, double *dL_dphi0, double *dL_dsigma,
                           double *dL_dM)
{
    if (!h) return LBM_ERR_ARG;
    if (!h->adj || !h->adj->ready) return afail(h, LBM_ERR_STATE, "lbm_adjoint_end needs lbm_adjoint_begin first");
    if (!dL_dphi) return afail(h, LBM_ERR_ARG, "dL_dphi must be non-NULL");
    lbm_status st = h->grid.precision == LBM_FP64 ? run_reverse<double>(h, dL_dphi, dL_dphi0, dL_dsigma, dL_dM)
                                                  : run_reverse<float>(h, dL_dphi, dL_dphi0, dL_dsigma, dL_dM);
    return st;
}

}  // extern "C"
