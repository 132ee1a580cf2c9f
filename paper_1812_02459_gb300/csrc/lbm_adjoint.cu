// lbm_adjoint.cu -- hand-written discrete adjoint of the lattice update.
//
// The reverse sweep works on a tape of plane operations.  To differentiate
// one step, the step is re-expressed as a sequence of whole-plane
// operations -- linear combinations, products, quotients, cubes, square
// roots, the clamp of rho(phi), stencils (isotropic gradient and Laplacian,
// fourth-order differences, the selective filter, the streaming shifts and
// bounce-back masks) and scalings by the differentiable parameters kappa,
// beta, M and 1/tau_f -- and recorded.  Each operation has a hand-written
// vector-Jacobian product; the reverse sweep applies them in reverse order.
// The operations run a level at a time: the stencils and pointwise
// operations between two layers of stencils form one kernel that applies
// them node by node, so a step costs one launch per level in each
// direction.  The schedule of a tape (levels, per-thread slots, flushes) is
// written out as straight-line CUDA C++ and compiled at run time (lbm_jit.h);
// interpreter kernels that read the same schedule from operation records are
// the fallback.  Across steps, sqrt(N)-style checkpointing keeps every k-th
// state, regenerates a segment with the fused forward kernels and reverses
// it step by step, the tape's forward passes of a segment batched and
// overlapped with the reverse passes on a second stream.  FP64 or FP32
// populations; the reverse sweep runs in the handle's arithmetic type, with
// the parameter gradients summed in FP64.  Walls (axes that are not
// periodic) as in the forward step: each stencil records the parity of its
// input along each axis, and across a wall it reads the mirror image about
// the halfway wall times that parity; streaming pulls from across a wall
// through a bounce-back mask stencil.  Walled tapes run on the compiled level
// kernels only (the interpreter's stencils are periodic).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <initializer_list>
#include <map>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_jit.h"

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
    // a mask stencil passes its one tap (0, 0) only where (x + mx, y + my)
    // lies across a wall (the bounce-back part of streaming)
    bool mask = false;
    int mx = 0, my = 0;
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
    // a stencil's ghost signs across a wall along x and y: the input's parity
    // (+1 even, -1 odd) in that direction, or 0 for a ghost that is zero
    signed char sgx = 1, sgy = 1;
};


// ---------------------------------------------------------------------------
// Execution of a recorded tape.  A plane's level counts the stencils on the
// longest path from the leaves to it.  Forward, one kernel per level: a
// thread takes a node, gathers the level's stencils from the (complete)
// planes of lower levels, then applies the level's pointwise operations in
// tape order.  Reverse, one kernel per level from the top: a thread takes a
// node, gathers the transposes of the next level's stencils from their
// (complete) output adjoints, then applies the vector-Jacobian products of
// the level's pointwise operations in reverse tape order.  Values made and
// used inside a kernel live in per-thread shared-memory slots, allocated by
// lifetime, and so do the adjoints accumulated inside a reverse kernel;
// other planes go through global memory.  The first contribution to each
// adjoint stores instead of adding, so nothing needs clearing.
// ---------------------------------------------------------------------------
int blocks_for(long long N) { return (int)std::min<long long>((N + NTH - 1) / NTH, 4096); }

#define GRID_LOOP(k, N) for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (N); \
                             k += (long long)gridDim.x * blockDim.x)

template <typename T> struct VOp {   // one operation as the level kernels run it
    int k, nin, param, live, st;
    int sgx, sgy;           // a stencil's ghost signs across walls (Op::sgx, Op::sgy)
    unsigned fint;          // bit i: input i is read from forward slot fslot[i]
    unsigned rassign;       // bit i: the contribution to reverse slot rslot[i] stores instead of adding
    short fslot[MAXIN], rslot[MAXIN];
    short fout, rout;       // forward slot of the output; reverse slot with its in-kernel adjoint (-1: none)
    T *out;                 // global plane of the output (null: not needed outside its kernel)
    const T *in[MAXIN];     // global planes of the inputs' values
    T c[MAXIN];
    T c0;                   // OP_LIN constant; OP_SCALEP parameter value
    const T *aout;          // global adjoint of the output (null: none reaches it from outside)
};
template <typename T> struct VFlush {   // end of a reverse kernel: dst (=) += slot
    T *dst;
    int slot, assign;
};
// One live operation of a reverse kernel, in execution order.  Every global
// value it reads was staged into a slot beforehand by a prefetch entry.
template <typename T> struct VRop {
    int k, nc, param, st;   // kind, contributions, parameter, stencil
    unsigned rassign;       // bit i: contribution i stores to its slot instead of adding
    short rslot[MAXIN];     // slot receiving contribution i
    short rout;             // slot with the in-kernel adjoint of the output (-1: none)
    short sa, sb, sz, sg;   // staged slots of in[0], in[1], out values and the outer output adjoint (-1: none)
    short stap;             // first staged slot of a stencil's taps (transpose gather)
    T c[MAXIN];
    T c0;
};
// A global value staged into slot `slot` ahead of use: p[voff + k] for a
// value plane, else p at the periodic neighbour (x + dx, y + dy).
template <typename T> struct VPre {
    const T *p;
    short slot;
    signed char dx, dy;
    int val;
};
// Reverse phase: ops [o0, o0 + no) run once entries [e0, e0 + ne) have landed.
struct VPhase { int o0, no, e0, ne; };
template <typename T> struct DW {   // a stencil's taps' weights in T
    int n;
    T w[MAXST];
};
// records are copied to shared memory in 8-byte words
static_assert(sizeof(VRop<float>) % 8 == 0 && sizeof(VRop<double>) % 8 == 0, "VRop size");
static_assert(sizeof(VPre<float>) % 8 == 0 && sizeof(VPre<double>) % 8 == 0, "VPre size");
static_assert(sizeof(DW<float>) % 8 == 0 && sizeof(DW<double>) % 8 == 0, "DW size");
static_assert(sizeof(VPhase) % 8 == 0, "VPhase size");
struct DStencil {
    int n;
    int dx[MAXST], dy[MAXST];
    double w[MAXST];
};
constexpr int MAXLEAF = 32;
template <typename T> struct Leaves {   // dst[i] = src[i] (floats or T), += with add, 0 with zero
    int n;
    T *dst[MAXLEAF];
    const void *src[MAXLEAF];
    unsigned f32, add, zero;
};

template <typename T> __device__ __forceinline__ void put(T *p, long long k, T v, bool assign)
{
    if (assign) p[k] = v;
    else p[k] += v;
}

// For B consecutive steps: dst[i][b N + k] (op)= src[i][b sstride + k].
template <typename T>
__global__ void __launch_bounds__(NTH) kk_leaves(Leaves<T> L, long long N, int B, long long sstride)
{
    GRID_LOOP(k, N * B) {
        const long long b = k / N, s = b * sstride + (k - b * N);
        for (int i = 0; i < L.n; ++i) {
            T v = T(0);
            if (!((L.zero >> i) & 1u))
                v = ((L.f32 >> i) & 1u) ? (T)((const float *)L.src[i])[s] : ((const T *)L.src[i])[s];
            put(L.dst[i], k, v, !((L.add >> i) & 1u));
        }
    }
}

constexpr int NTV = 128;   // threads of an interpreter level kernel

// Copy records (8-byte aligned) into shared memory; every thread of the
// block takes part and the block waits for the copy.
__device__ __forceinline__ void stage_records(void *dst, const void *src, size_t bytes)
{
    unsigned long long *d = reinterpret_cast<unsigned long long *>(dst);
    const unsigned long long *s = reinterpret_cast<const unsigned long long *>(src);
    for (size_t i = threadIdx.x; i < bytes / 8; i += blockDim.x) d[i] = s[i];
    __syncthreads();
}

// Shared memory of a level kernel: the stencil table, the kernel's
// operation records, then the slots (NTV values per slot).
template <typename T> struct VmLayout {
    static __host__ __device__ size_t tab_bytes(int ntab) { return (sizeof(DStencil) * (size_t)ntab + 15) / 16 * 16; }
    static __host__ __device__ size_t ops_bytes(int nops) { return (sizeof(VOp<T>) * (size_t)nops + 15) / 16 * 16; }
    static __host__ __device__ size_t bytes(int ntab, int nops, int slots)
    {
        return tab_bytes(ntab) + ops_bytes(nops) + sizeof(T) * NTV * (size_t)slots;
    }
};

template <typename T> __device__ __forceinline__ T &slot_ref(T *sl, int q) { return sl[q * NTV + threadIdx.x]; }

// sum_i w_i src(x + sg dx_i, y + sg dy_i) over the n <= NB taps of S on the
// periodic grid, every tap requested before the first is used (|d| <= 5).
template <typename T, int NB>
__device__ __forceinline__ T taps(const DStencil &S, const T *src, int x, int y, int sg, int nx, int ny)
{
    const int n = S.n;
    T v[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) {
        if (i < n) {
            int xx = x + sg * S.dx[i], yy = y + sg * S.dy[i];
            xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
            yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
            v[i] = src[(long long)yy * nx + xx];
        }
    }
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < NB; ++i)
        if (i < n) acc += (T)S.w[i] * v[i];
    return acc;
}
template <typename T>
__device__ __forceinline__ T gather(const DStencil &S, const T *src, int x, int y, int sg, int nx, int ny)
{
    return S.n <= 1 ? taps<T, 1>(S, src, x, y, sg, nx, ny)
                    : (S.n <= 9 ? taps<T, 9>(S, src, x, y, sg, nx, ny) : taps<T, MAXST>(S, src, x, y, sg, nx, ny));
}

template <typename T>
__global__ void __launch_bounds__(NTV) kk_vm_fwd(const DStencil *__restrict__ gtab, int ntab,
                                                const VOp<T> *__restrict__ gops, int nops, int nx, int ny, long long N,
                                                long long Ntot, long long voff)
{
    // Ntot = B N nodes of B consecutive steps, whose values sit from offset
    // voff in the value planes
    extern __shared__ __align__(16) unsigned char vm_raw[];
    using Ly = VmLayout<T>;
    DStencil *tab = reinterpret_cast<DStencil *>(vm_raw);
    VOp<T> *ops = reinterpret_cast<VOp<T> *>(vm_raw + Ly::tab_bytes(ntab));
    T *sl = reinterpret_cast<T *>(vm_raw + Ly::tab_bytes(ntab) + Ly::ops_bytes(nops));
    stage_records(tab, gtab, sizeof(DStencil) * (size_t)ntab);
    stage_records(ops, gops, sizeof(VOp<T>) * (size_t)nops);
    GRID_LOOP(k, Ntot) {
        const long long base = (k / N) * N, kk = k - base;
        const int y = (int)(kk / nx), x = (int)(kk - (long long)y * nx);
        for (int o = 0; o < nops; ++o) {
            const VOp<T> &op = ops[o];
            T r;
            if (op.k == OP_STENCIL) {
                r = gather(tab[op.st], op.in[0] + voff + base, x, y, 1, nx, ny);
            } else {
                const int nin = op.nin;
                T v[MAXIN];
#pragma unroll
                for (int i = 0; i < MAXIN; ++i)   // every input requested before the first is used
                    if (i < nin) v[i] = ((op.fint >> i) & 1u) ? slot_ref(sl, op.fslot[i]) : op.in[i][voff + k];
                switch (op.k) {
                case OP_LIN:
                    r = op.c0;
#pragma unroll
                    for (int i = 0; i < MAXIN; ++i)
                        if (i < nin) r += op.c[i] * v[i];
                    break;
                case OP_SCALEP: r = op.c0 * v[0]; break;
                case OP_MUL: r = v[0] * v[1]; break;
                case OP_DIV: r = v[0] / v[1]; break;
                case OP_POW3: r = v[0] * v[0] * v[0]; break;
                case OP_SQRT: r = sqrt(v[0]); break;
                case OP_CLAMP1: r = v[0] < T(-1) ? T(-1) : (v[0] > T(1) ? T(1) : v[0]); break;
                default: r = T(1) / v[0]; break;   // OP_RECIP
                }
            }
            if (op.fout >= 0) slot_ref(sl, op.fout) = r;
            if (op.out) op.out[voff + k] = r;
        }
    }
}

// Asynchronous 4- or 8-byte copy global -> shared (cp.async, sm_80 and
// later); the issuing thread waits for its own groups.
template <typename T> __device__ __forceinline__ void cp_async_val(T *dst, const T *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (sizeof(T) == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int NW> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(NW) : "memory"); }

// Shared memory of a reverse kernel: tap weights, operation records,
// prefetch entries, phases, flushes, then the slots (NTV values per slot).
template <typename T> struct RevLayout {
    static __host__ __device__ size_t al(size_t b) { return (b + 15) / 16 * 16; }
    static __host__ __device__ size_t w(int ntab) { return al(sizeof(DW<T>) * (size_t)ntab); }
    static __host__ __device__ size_t o(int nops) { return al(sizeof(VRop<T>) * (size_t)nops); }
    static __host__ __device__ size_t e(int npre) { return al(sizeof(VPre<T>) * (size_t)npre); }
    static __host__ __device__ size_t p(int nph) { return al(sizeof(VPhase) * (size_t)nph); }
    static __host__ __device__ size_t f(int nfl) { return al(sizeof(VFlush<T>) * (size_t)nfl); }
    static __host__ __device__ size_t bytes(int ntab, int nops, int npre, int nph, int nfl, int slots)
    {
        return w(ntab) + o(nops) + e(npre) + p(nph) + f(nfl) + sizeof(T) * NTV * (size_t)slots;
    }
};

// Records of one reverse kernel (device pointers into the engine's arrays).
template <typename T> struct RevArgs {
    const DW<T> *tw;
    const VRop<T> *ops;
    const VPre<T> *pre;
    const VPhase *ph;
    const VFlush<T> *fl;
    int ntab, nops, npre, nph, nfl;
};

template <typename T>
__global__ void __launch_bounds__(NTV) kk_vm_rev(RevArgs<T> A, double *pgrad, int nx, int ny, long long N,
                                                long long voff)
{
    // The forward values of the step are at offset voff in the value planes.
    // A node's global reads are staged into slots a phase ahead of the ops
    // that use them (two staging buffers alternate), so a phase's loads are
    // in flight while the previous phase computes.  Every contribution goes
    // to a slot; the slots holding the adjoints of planes outside the kernel
    // are flushed at the end.
    extern __shared__ __align__(16) unsigned char vm_raw[];
    using Ly = RevLayout<T>;
    unsigned char *q = vm_raw;
    DW<T> *tw = reinterpret_cast<DW<T> *>(q); q += Ly::w(A.ntab);
    VRop<T> *ops = reinterpret_cast<VRop<T> *>(q); q += Ly::o(A.nops);
    VPre<T> *pre = reinterpret_cast<VPre<T> *>(q); q += Ly::e(A.npre);
    VPhase *ph = reinterpret_cast<VPhase *>(q); q += Ly::p(A.nph);
    VFlush<T> *fl = reinterpret_cast<VFlush<T> *>(q); q += Ly::f(A.nfl);
    T *sl = reinterpret_cast<T *>(q);
    stage_records(tw, A.tw, sizeof(DW<T>) * (size_t)A.ntab);
    stage_records(ops, A.ops, sizeof(VRop<T>) * (size_t)A.nops);
    stage_records(pre, A.pre, sizeof(VPre<T>) * (size_t)A.npre);
    stage_records(ph, A.ph, sizeof(VPhase) * (size_t)A.nph);
    stage_records(fl, A.fl, sizeof(VFlush<T>) * (size_t)A.nfl);
    const int nph = A.nph, nfl = A.nfl;
    double pacc[NPARAM] = {};
    GRID_LOOP(k, N) {
        const int y = (int)(k / nx), x = (int)(k - (long long)y * nx);
        auto issue = [&](int p) {
            const VPhase P = ph[p];
            for (int e = P.e0; e < P.e0 + P.ne; ++e) {
                const VPre<T> E = pre[e];
                const T *src;
                if (E.val) src = E.p + voff + k;
                else {
                    int xx = x + E.dx, yy = y + E.dy;
                    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
                    yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
                    src = E.p + (long long)yy * nx + xx;
                }
                cp_async_val(&slot_ref(sl, E.slot), src);
            }
            cp_async_commit();
        };
        if (nph > 0) issue(0);
        for (int p = 0; p < nph; ++p) {
            if (p + 1 < nph) {
                issue(p + 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            const VPhase P = ph[p];
            for (int o = P.o0; o < P.o0 + P.no; ++o) {
                const VRop<T> &op = ops[o];
                const int kind = op.k;
                T ci[MAXIN];
                const int nc = op.nc;
                if (kind == OP_STENCIL) {   // transpose: the staged taps of the output adjoint around the node
                    const DW<T> &W = tw[op.st];
                    T acc = T(0);
                    for (int j = 0; j < W.n; ++j) acc += W.w[j] * slot_ref(sl, op.stap + j);
                    ci[0] = acc;
                } else {
                    const T a = op.sa >= 0 ? slot_ref(sl, op.sa) : T(0);
                    const T b = op.sb >= 0 ? slot_ref(sl, op.sb) : T(0);
                    const T z = op.sz >= 0 ? slot_ref(sl, op.sz) : T(0);
                    T g = op.sg >= 0 ? slot_ref(sl, op.sg) : T(0);
                    if (op.rout >= 0) g += slot_ref(sl, op.rout);
                    switch (kind) {
                    case OP_LIN:
#pragma unroll
                        for (int i = 0; i < MAXIN; ++i) ci[i] = op.c[i] * g;
                        break;
                    case OP_SCALEP: {
                        ci[0] = op.c0 * g;
                        const double d = (double)a * (double)g;
#pragma unroll
                        for (int q = 0; q < NPARAM; ++q) pacc[q] += q == op.param ? d : 0.0;
                        break;
                    }
                    case OP_MUL: ci[0] = b * g; ci[1] = a * g; break;
                    case OP_DIV: ci[0] = g / b; ci[1] = -(g * a / (b * b)); break;
                    case OP_POW3: ci[0] = T(3) * a * a * g; break;
                    case OP_SQRT: ci[0] = g / (T(2) * z); break;
                    case OP_CLAMP1: ci[0] = (a >= T(-1) && a <= T(1)) ? g : T(0); break;
                    default: ci[0] = -(g / (a * a)); break;   // OP_RECIP
                    }
                }
#pragma unroll
                for (int i = 0; i < MAXIN; ++i) {
                    if (i >= nc) break;
                    T &r = slot_ref(sl, op.rslot[i]);
                    r = ((op.rassign >> i) & 1u) ? ci[i] : r + ci[i];
                }
            }
        }
        constexpr int FB = 8;   // flushes whose old values are requested together
        for (int f0 = 0; f0 < nfl; f0 += FB) {
            T old[FB];
#pragma unroll
            for (int i = 0; i < FB; ++i) {
                old[i] = T(0);
                if (f0 + i < nfl && !fl[f0 + i].assign) old[i] = fl[f0 + i].dst[k];
            }
#pragma unroll
            for (int i = 0; i < FB; ++i)
                if (f0 + i < nfl) fl[f0 + i].dst[k] = old[i] + slot_ref(sl, fl[f0 + i].slot);
        }
    }
    __shared__ double red[NPARAM][NTV / 32];
#pragma unroll
    for (int q = 0; q < NPARAM; ++q) {
        double v = pacc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < NPARAM) {
        double t = 0.0;
        for (int w = 0; w < NTV / 32; ++w) t += red[threadIdx.x][w];
        if (t != 0.0) atomicAdd(pgrad + threadIdx.x, t);
    }
}

// ---------------------------------------------------------------------------
// The tape engine.  Planes are kept per plane id across steps (the recorder
// creates the same planes in the same order every step), so the schedule
// and the device form of the tape are built once and reused while the
// recorded tape stays the same.
// ---------------------------------------------------------------------------
template <typename T> struct Engine {
    int nx = 0, ny = 0;
    int perx = 1, pery = 1;           // periodic axes; a wall stands halfway beyond the edge of the others
    bool walls() const { return !perx || !pery; }
    long long N = 0;
    cudaStream_t st = nullptr;        // forward passes
    cudaStream_t rst = nullptr;       // reverse passes and collection (st when null)
    cudaError_t err = cudaSuccess;
    std::vector<T *> val, adj;        // by plane id, persistent; a value plane holds nvbuf buffers of Bcap steps
    int nval = 0;
    int Bwant = 1, Bcap = 0;          // steps wanted in one forward batch; steps one value buffer holds
    int nvbuf = 1;                    // value buffers: with two, a batch's forward pass can run while
                                      // the reverse pass of the previous batch reads the other buffer
    long long leaf_stride = 0;        // elements between two consecutive steps' leaf sources
    std::vector<Op> tape;
    std::vector<Stencil> stencils;
    double pval[NPARAM]{};
    double *d_pgrad = nullptr;
    int nb = 1;
    std::vector<std::pair<int, const void *>> leaves;   // plane, source (this step)
    std::vector<char> leaf_f32;
    std::vector<std::pair<int, const T *>> seeds;       // plane, adjoint source
    std::vector<char> flowed;                           // planes given a global adjoint by run()
    // schedule and device form
    struct Group { int off, n, slots; };
    struct RGroup { int op0, nops, pre0, npre, ph0, nph, fl0, nfl, slots; };
    std::vector<Group> fgroups;                         // launch order
    std::vector<RGroup> rgroups;
    std::vector<VOp<T>> hfwd;
    std::vector<VRop<T>> hrop;
    std::vector<VPre<T>> hpre;
    std::vector<VPhase> hph;
    std::vector<VFlush<T>> hfl;
    VOp<T> *d_fwd = nullptr;
    VRop<T> *d_rop = nullptr;
    VPre<T> *d_pre = nullptr;
    VPhase *d_ph = nullptr;
    VFlush<T> *d_fl = nullptr;
    DW<T> *d_tw = nullptr;
    size_t cap_fwd = 0, cap_rop = 0, cap_pre = 0, cap_ph = 0, cap_fl = 0;
    static constexpr int STAGE = 16;                    // staged loads per reverse phase (more for a wide stencil)
    // compiled level kernels: the schedule written out as straight-line
    // CUDA C++ (one kernel per level and direction), plane pointers and
    // coefficients passed in one argument struct
    struct JKernel { cudaKernel_t k = nullptr; std::vector<unsigned long long> pack, pack_sw; int np = 0; };
    std::vector<JKernel> jfwd, jrev;
    bool jit = false;                                   // the compiled kernels run the scheduled tape
    bool pingpong = false;                              // reverse packs with the state adjoints exchanged exist
    static constexpr int JTY = 4;                       // compiled kernels: a block is a tile of 32 x JTY nodes
    static constexpr int JT = 32 * JTY;                 // threads of a compiled level kernel
    static std::string bounds() { return "__launch_bounds__(" + std::to_string(JT) + ", " + std::to_string(512 / JT) + ")"; }
    DStencil *d_tab = nullptr;
    int ntab = 0, nbv = 1;
    int smem_set = 0;
    std::vector<Op> tape_prev;
    std::vector<std::pair<int, const T *>> seeds_prev;
    std::vector<char> seed_add;

    void check(cudaError_t e) { if (e != cudaSuccess && err == cudaSuccess) err = e; }

    std::vector<void *> val_chunks, adj_chunks;   // planes are carved from a few allocations
    // Give each plane ids[j] without storage its own elems-element slice
    // (256-byte aligned) of one new allocation.
    void carve(std::vector<T *> &planes, const std::vector<int> &ids, size_t elems, std::vector<void *> &chunks)
    {
        if (ids.empty()) return;
        const size_t stride = (sizeof(T) * elems + 255) / 256 * 256;
        void *b = nullptr;
        check(cudaMalloc(&b, stride * ids.size()));
        if (err != cudaSuccess) return;
        chunks.push_back(b);
        for (size_t j = 0; j < ids.size(); ++j) planes[ids[j]] = (T *)((char *)b + stride * j);
    }
    void free_chunks(std::vector<void *> &chunks)
    {
        for (void *b : chunks) cudaFree(b);
        chunks.clear();
    }
    void reset()
    {
        nval = 0;
        tape.clear();
        leaves.clear();
        leaf_f32.clear();
        seeds.clear();
    }
    void release_all()
    {
        free_chunks(val_chunks);
        free_chunks(adj_chunks);
        val.clear();
        adj.clear();
        nval = 0;
        Bcap = 0;
        nvbuf = 1;
        void *bufs[8] = {d_pgrad, d_fwd, d_rop, d_pre, d_ph, d_fl, d_tab, d_tw};
        for (void *b : bufs) if (b) cudaFree(b);
        d_pgrad = nullptr;
        d_fwd = nullptr;
        d_rop = nullptr;
        d_pre = nullptr;
        d_ph = nullptr;
        d_fl = nullptr;
        d_tab = nullptr;
        d_tw = nullptr;
        cap_fwd = cap_rop = cap_pre = cap_ph = cap_fl = 0;
        tape_prev.clear();
    }
    int newplane()   // value planes are allocated by schedule(), once the batch size is known
    {
        if (nval == (int)val.size()) {
            val.push_back(nullptr);
            adj.push_back(nullptr);
        }
        return nval++;
    }
    // Value planes (those with stored[p] set) of nvbuf buffers of B steps
    // each, within a quarter of the free device memory: two
    // buffers when two steps fit, B = Bwant or as many as fit.  The buffer
    // count is fixed at the first sizing after release_all().
    void size_values(const std::vector<char> &stored)
    {
        size_t fr = 0, tot = 0;
        check(cudaMemGetInfo(&fr, &tot));
        const double nst = (double)std::count(stored.begin(), stored.end(), 1);
        const double per_step = (double)sizeof(T) * (double)N * nst;
        const double budget = (double)fr / 4.0;
        if (Bcap == 0) nvbuf = 2.0 * per_step <= budget ? 2 : 1;
        const int B = std::max(1, std::min(Bwant, (int)(budget / std::max(per_step * nvbuf, 1.0))));
        if (B > Bcap) {
            free_chunks(val_chunks);
            std::fill(val.begin(), val.end(), nullptr);
            Bcap = B;
        }
        std::vector<int> need;
        for (int i = 0; i < nval; ++i)
            if (stored[i] && !val[i]) need.push_back(i);
        carve(val, need, (size_t)N * Bcap * nvbuf, val_chunks);
    }
    long long vbase(int vb) const { return (long long)vb * Bcap * N; }   // start of value buffer vb
    // Value plane of leaf i for step j of value buffer vb.
    T *leaf_dst(int i, int vb, int j) { return val[leaves[i].first] + vbase(vb) + (long long)j * N; }
    template <typename U> int leaf(const U *src)
    {
        static_assert(sizeof(U) == sizeof(T) || sizeof(U) == sizeof(float), "leaf type");
        int id = newplane();
        leaves.push_back({id, (const void *)src});
        leaf_f32.push_back(sizeof(U) == sizeof(float) && sizeof(T) != sizeof(float));
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
    // a stencil on plane a; across a wall the ghosts are the mirror images
    // about the halfway wall times sgx (x) and sgy (y)
    int sten(int a, int s, int sgx = 1, int sgy = 1)
    {
        Op o;
        o.k = OP_STENCIL;
        o.in[0] = a;
        o.nin = 1;
        o.st = s;
        o.sgx = (signed char)sgx;
        o.sgy = (signed char)sgy;
        return emit(o);
    }
    int scalep(int a, int p) { Op o; o.k = OP_SCALEP; o.in[0] = a; o.nin = 1; o.param = p; return emit(o); }
    int emit(Op o)
    {
        o.out = newplane();
        tape.push_back(o);
        return o.out;
    }
    void seed(int id, const T *src) { seeds.push_back({id, src}); }

    static bool same_tape(const std::vector<Op> &a, const std::vector<Op> &b)
    {
        if (a.size() != b.size()) return false;
        for (size_t i = 0; i < a.size(); ++i) {
            const Op &x = a[i], &y = b[i];
            if (x.k != y.k || x.out != y.out || x.nin != y.nin || x.c0 != y.c0 || x.param != y.param || x.st != y.st ||
                x.sgx != y.sgx || x.sgy != y.sgy)
                return false;
            for (int j = 0; j < x.nin; ++j)
                if (x.in[j] != y.in[j] || x.c[j] != y.c[j]) return false;
        }
        return true;
    }

    // Build the schedule of the recorded tape unless it is the one built last.
    void prepare()
    {
        if (!(same_tape(tape, tape_prev) && seeds == seeds_prev)) schedule();
    }
    // Forward and reverse sweep of a single step (leaf sources as recorded).
    void run()
    {
        prepare();
        if (err != cudaSuccess) return;
        forward(0, 1);
        reverse(0);
    }

    static int ncontrib(const Op &o)   // inputs an operation's product reaches
    {
        return o.k == OP_LIN ? o.nin : (o.k == OP_MUL || o.k == OP_DIV) ? 2 : 1;
    }

    void schedule()
    {
        const int nops = (int)tape.size();
        ntab = (int)stencils.size();
        std::vector<int> lev(nval, -1), made(nval, -1);   // level of a plane (-1: leaf); op making it
        int L = 0;
        for (int t = 0; t < nops; ++t) {
            const Op &o = tape[t];
            int l = 0;
            for (int i = 0; i < o.nin; ++i) l = std::max(l, std::max(lev[o.in[i]], 0));
            if (o.k == OP_STENCIL) ++l;
            lev[o.out] = l;
            made[o.out] = t;
            L = std::max(L, l);
        }
        // kernel lists: forward F_l = stencils of level l, then pointwise ops
        // of level l (tape order); reverse R_l = pointwise ops of level l, then
        // stencils of level l + 1 (walked from the end)
        std::vector<std::vector<int>> F(L + 1), R(L + 1);
        for (int t = 0; t < nops; ++t)
            if (tape[t].k == OP_STENCIL) F[lev[tape[t].out]].push_back(t);
        for (int t = 0; t < nops; ++t)
            if (tape[t].k != OP_STENCIL) F[lev[tape[t].out]].push_back(t);
        for (int t = 0; t < nops; ++t)
            if (tape[t].k != OP_STENCIL) R[lev[tape[t].out]].push_back(t);
        for (int t = 0; t < nops; ++t)
            if (tape[t].k == OP_STENCIL) R[lev[tape[t].out] - 1].push_back(t);
        // a value is inside forward kernel l when made there; inside reverse
        // kernel l when made by a pointwise op of level l (stencil outputs
        // keep global adjoints: their transposes gather them around a node)
        auto fin_kernel = [&](int p) { return made[p] >= 0 ? lev[p] : -1; };
        auto rin_kernel = [&](int p) { return (made[p] >= 0 && tape[made[p]].k != OP_STENCIL) ? lev[p] : -1; };
        std::vector<char> used_out(nval, 0), needs_val(nval, 0);
        for (int t = 0; t < nops; ++t) {
            const Op &o = tape[t];
            for (int i = 0; i < o.nin; ++i)
                if (o.k == OP_STENCIL || fin_kernel(o.in[i]) != lev[o.out]) used_out[o.in[i]] = 1;
            if (o.k == OP_MUL || o.k == OP_DIV) needs_val[o.in[0]] = needs_val[o.in[1]] = 1;
            if (o.k == OP_POW3 || o.k == OP_CLAMP1 || o.k == OP_RECIP || o.k == OP_SCALEP) needs_val[o.in[0]] = 1;
            if (o.k == OP_SQRT) needs_val[o.out] = 1;
        }
        // planes kept in global memory: the leaves, planes read outside the
        // forward kernel making them, and values the reverse sweep reads
        std::vector<char> stored(nval, 0);
        for (int p = 0; p < nval; ++p) stored[p] = made[p] < 0 || used_out[p] || needs_val[p];
        size_values(stored);
        if (err != cudaSuccess) return;
        // the reverse sweep, simulated in execution order
        std::vector<char> gw(nval, 0), init(nval, 0);
        seed_add.assign(seeds.size(), 0);
        for (size_t i = 0; i < seeds.size(); ++i) {
            seed_add[i] = init[seeds[i].first];
            gw[seeds[i].first] = init[seeds[i].first] = 1;
        }
        std::vector<VOp<T>> rec(nops);
        for (int t = 0; t < nops; ++t) {
            rec[t] = VOp<T>{};
            rec[t].fout = rec[t].rout = -1;
        }
        // adjoints of planes outside a reverse kernel are collected in slots
        // too and flushed to global memory once, at the kernel's end
        std::vector<int> rslots(L + 1, 0), rslotof(nval, -1), gslotof(nval, -1);
        std::vector<std::vector<std::pair<int, int>>> flush(L + 1);   // plane, slot
        std::vector<std::vector<char>> flush_as(L + 1);
        for (int l = L; l >= 0; --l) {
            std::vector<int> freel;
            int top = 0;
            auto alloc = [&]() { if (!freel.empty()) { int q = freel.back(); freel.pop_back(); return q; } return top++; };
            for (int j = (int)R[l].size() - 1; j >= 0; --j) {
                const int t = R[l][j];
                const Op &o = tape[t];
                VOp<T> &d = rec[t];
                const bool inner = rslotof[o.out] >= 0;
                if (!gw[o.out] && !inner) continue;
                d.live = 1;
                if (inner) {
                    d.rout = (short)rslotof[o.out];
                    freel.push_back(rslotof[o.out]);
                    rslotof[o.out] = -1;
                }
                for (int i = 0; i < ncontrib(o); ++i) {
                    const int p = o.in[i];
                    if (rin_kernel(p) == l) {
                        if (rslotof[p] < 0) { rslotof[p] = alloc(); d.rassign |= 1u << i; }
                        d.rslot[i] = (short)rslotof[p];
                    } else {
                        if (gslotof[p] < 0) {
                            gslotof[p] = alloc();
                            d.rassign |= 1u << i;
                            flush[l].push_back({p, gslotof[p]});
                        }
                        d.rslot[i] = (short)gslotof[p];
                    }
                }
            }
            for (auto &f : flush[l]) {
                flush_as[l].push_back(!init[f.first]);
                gw[f.first] = init[f.first] = 1;
                gslotof[f.first] = -1;
            }
            rslots[l] = top;
        }
        std::vector<int> need;
        for (int p = 0; p < nval; ++p)
            if (gw[p] && !adj[p]) need.push_back(p);
        carve(adj, need, (size_t)N, adj_chunks);
        if (err != cudaSuccess) return;
        flowed = gw;
        // forward slots and the rest of each record
        std::vector<int> fslots(L + 1, 0), fslotof(nval, -1), lastuse(nval, -1);
        for (int l = 0; l <= L; ++l) {
            for (size_t j = 0; j < F[l].size(); ++j) {
                const Op &o = tape[F[l][j]];
                for (int i = 0; i < o.nin; ++i)
                    if (fin_kernel(o.in[i]) == l && o.k != OP_STENCIL) lastuse[o.in[i]] = (int)j;
            }
            std::vector<int> freel;
            int top = 0;
            for (size_t j = 0; j < F[l].size(); ++j) {
                const int t = F[l][j];
                const Op &o = tape[t];
                VOp<T> &d = rec[t];
                d.k = o.k;
                d.nin = o.nin;
                d.param = o.param;
                d.st = o.st;
                d.sgx = o.sgx;
                d.sgy = o.sgy;
                for (int i = 0; i < o.nin; ++i) {
                    const int p = o.in[i];
                    d.in[i] = val[p];
                    d.c[i] = (T)o.c[i];
                    if (o.k != OP_STENCIL && fin_kernel(p) == l) {
                        d.fint |= 1u << i;
                        d.fslot[i] = (short)fslotof[p];
                    }
                }
                for (int i = 0; i < o.nin; ++i) {   // inputs read for the last time free their slots
                    const int p = o.in[i];
                    if (o.k != OP_STENCIL && fin_kernel(p) == l && lastuse[p] == (int)j && fslotof[p] >= 0) {
                        freel.push_back(fslotof[p]);
                        fslotof[p] = -1;
                    }
                }
                if (lastuse[o.out] > (int)j) {
                    int q;
                    if (!freel.empty()) { q = freel.back(); freel.pop_back(); } else q = top++;
                    fslotof[o.out] = q;
                    d.fout = (short)q;
                }
                d.out = (used_out[o.out] || needs_val[o.out]) ? val[o.out] : nullptr;
                d.c0 = o.k == OP_SCALEP ? (T)pval[o.param] : (T)o.c0;
                d.aout = (d.live && gw[o.out]) ? adj[o.out] : nullptr;
            }
            fslots[l] = top;
        }
        // device form in launch order
        hfwd.clear();
        hrop.clear();
        hpre.clear();
        hph.clear();
        hfl.clear();
        fgroups.clear();
        rgroups.clear();
        int smem = 0;
        for (int l = 0; l <= L; ++l) {
            if (F[l].empty()) continue;
            fgroups.push_back({(int)hfwd.size(), (int)F[l].size(), fslots[l]});
            for (int t : F[l]) hfwd.push_back(rec[t]);
            smem = std::max(smem, (int)VmLayout<T>::bytes(ntab, (int)F[l].size(), fslots[l]));
        }
        std::vector<std::vector<int>> rex;   // per reverse group: its live operations in execution order
        for (int l = L; l >= 0; --l) {
            std::vector<int> ex;   // live operations in execution order
            for (int j = (int)R[l].size() - 1; j >= 0; --j)
                if (rec[R[l][j]].live) ex.push_back(R[l][j]);
            const int nfl = (int)flush[l].size();
            if (ex.empty() && nfl == 0) continue;
            add_rgroup(ex, rslots[l], rec);
            rex.push_back(ex);
            RGroup &G = rgroups.back();
            G.fl0 = (int)hfl.size();
            G.nfl = nfl;
            for (int i = 0; i < nfl; ++i)
                hfl.push_back({adj[flush[l][i].first], flush[l][i].second, flush_as[l][i] ? 1 : 0});
            smem = std::max(smem, (int)RevLayout<T>::bytes(ntab, G.nops, G.npre, G.nph, G.nfl, G.slots));
        }
        if (smem > smem_set) {
            check(cudaFuncSetAttribute(kk_vm_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            check(cudaFuncSetAttribute(kk_vm_rev<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
            smem_set = smem;
        }
        nbv = (int)std::min<long long>((N + NTV - 1) / NTV, 8192);
        compile_levels(rec, rex);
        upload();
        tape_prev = tape;
        seeds_prev = seeds;
    }

    // Arguments of one compiled kernel: distinct plane pointers, coefficients.
    struct ArgPack {
        std::vector<const void *> ptr;
        std::map<const void *, int> at;
        std::vector<T> coef;
        std::string p(const void *q)
        {
            auto it = at.find(q);
            if (it == at.end()) { it = at.emplace(q, (int)ptr.size()).first; ptr.push_back(q); }
            return "A.p[" + std::to_string(it->second) + "]";
        }
        std::string c(double v)
        {
            coef.push_back((T)v);
            return "A.c[" + std::to_string(coef.size() - 1) + "]";
        }
        std::string decl(const std::string &name) const
        {
            return "struct " + name + " { T *p[" + std::to_string(std::max<size_t>(1, ptr.size())) + "]; T c[" +
                   std::to_string(std::max<size_t>(1, coef.size())) + "]; };\n";
        }
        std::vector<unsigned long long> pack() const   // the struct's bytes
        {
            const size_t np = std::max<size_t>(1, ptr.size()), nc = std::max<size_t>(1, coef.size());
            std::vector<unsigned long long> w(np + (sizeof(T) * nc + 7) / 8, 0ull);
            std::memcpy(w.data(), ptr.data(), sizeof(void *) * ptr.size());
            std::memcpy((char *)w.data() + 8 * np, coef.data(), sizeof(T) * coef.size());
            return w;
        }
    };
    static std::string S(int i) { return std::to_string(i); }

    // Forward level kernel gi: the records of fgroups[gi] in order, a
    // thread per node of a batch of steps; slot q is the variable fq.
    // Global loads of a generated kernel, each (plane, tap) read once: the
    // first use declares a variable in the node loop's scope.
    struct Loads {
        std::map<std::pair<const void *, int>, std::string> at;
        std::string decl;   // declarations to emit before the current operation
        std::string get(ArgPack &A, const void *p, int dx, int dy, bool tap, const char *off)
        {
            const int key = tap ? (dx + 64) * 256 + (dy + 64) : -1;
            auto it = at.find({p, key});
            if (it != at.end()) return it->second;
            const std::string v = "g" + S((int)at.size());
            decl += "        const T " + v + " = __ldg(" + A.p(p) + " + " + off +
                    (tap ? " + nbi(x, y, " + S(dx) + ", " + S(dy) + ", nx, ny)" : std::string(" + k")) + ");\n";
            at.emplace(std::make_pair(p, key), v);
            return v;
        }
    };

    std::string gen_fwd(int gi, ArgPack &A)
    {
        const Group &G = fgroups[gi];
        std::string b;
        Loads ld;
        for (int j = 0; j < G.n; ++j) {
            const VOp<T> &d = hfwd[G.off + j];
            std::string o = "        {\n";
            if (d.k == OP_STENCIL && stencils[d.st].mask) {
                const Stencil &St = stencils[d.st];
                o += "            const T r = wout(x + " + S(St.mx) + ", y + " + S(St.my) + ", nx, ny) ? " +
                     ld.get(A, d.in[0], 0, 0, true, "voff + base") + " : T(0);\n";
            } else if (d.k == OP_STENCIL) {
                const Stencil &St = stencils[d.st];
                o += "            T r = T(0);\n";
                std::string plain;
                for (int i = 0; i < St.n; ++i)
                    plain += "            r += " + A.c(St.w[i]) + " * " +
                             ld.get(A, d.in[0], St.dx[i], St.dy[i], true, "voff + base") + ";\n";
                if (walls()) {   // interior nodes: every tap inside, no mirror
                    o += "            if (inner) {\n" + plain + "            } else {\n";
                    for (int i = 0; i < St.n; ++i)
                        o += "            r += " + A.c(St.w[i]) + " * wtap(" + A.p(d.in[0]) + " + voff + base, x, y, " +
                             S(St.dx[i]) + ", " + S(St.dy[i]) + ", nx, ny, T(" + S(d.sgx) + "), T(" + S(d.sgy) + "));\n";
                    o += "            }\n";
                } else {
                    o += plain;
                }
            } else {
                for (int i = 0; i < d.nin; ++i)
                    o += "            const T v" + S(i) + " = " +
                         (((d.fint >> i) & 1u) ? "f" + S(d.fslot[i]) : ld.get(A, d.in[i], 0, 0, false, "voff")) + ";\n";
                switch (d.k) {
                case OP_LIN:
                    o += "            T r = " + A.c((double)d.c0) + ";\n";
                    for (int i = 0; i < d.nin; ++i) o += "            r += " + A.c((double)d.c[i]) + " * v" + S(i) + ";\n";
                    break;
                case OP_SCALEP: o += "            const T r = " + A.c((double)d.c0) + " * v0;\n"; break;
                case OP_MUL: o += "            const T r = v0 * v1;\n"; break;
                case OP_DIV: o += "            const T r = v0 / v1;\n"; break;
                case OP_POW3: o += "            const T r = v0 * v0 * v0;\n"; break;
                case OP_SQRT: o += "            const T r = sqrt(v0);\n"; break;
                case OP_CLAMP1: o += "            const T r = v0 < T(-1) ? T(-1) : (v0 > T(1) ? T(1) : v0);\n"; break;
                default: o += "            const T r = T(1) / v0;\n"; break;   // OP_RECIP
                }
            }
            if (d.fout >= 0) o += "            f" + S(d.fout) + " = r;\n";
            if (d.out) o += "            " + A.p(d.out) + "[voff + k] = r;\n";
            b += ld.decl + o + "        }\n";
            ld.decl.clear();
        }
        std::string f = A.decl("KF" + S(gi));
        f += "extern \"C\" __global__ void " + bounds() + " f" + S(gi) +
             "(const KF" + S(gi) + " A, long long N, long long Ntot, long long voff, int nx, int ny)\n{\n"
             "    const long long tiles_x = (nx + 31) / 32, tpp = tiles_x * ((ny + JTY - 1) / JTY), ntiles = tpp * (Ntot / N);\n"
             "    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {\n"
             "        int x, y;\n"
             "        long long k;\n"
             "        if (!tile_node(t, tiles_x, tpp, nx, ny, N, x, y, k)) continue;\n"
             "        const long long base = k - ((long long)y * nx + x);\n" + inner_flag();
        for (int q = 0; q < G.slots; ++q) f += "        T f" + S(q) + " = T(0);\n";
        return f + b + "    }\n}\n";
    }

    // Reverse level kernel gi: the live operations ex in execution order,
    // a thread per node; accumulation slot q is the variable sq; the slots
    // of outer planes are flushed at the end.
    std::string gen_rev(int gi, const std::vector<int> &ex, const std::vector<VOp<T>> &rec, int nslots, ArgPack &A)
    {
        const RGroup &G = rgroups[gi];
        std::string b;
        bool pgr = false;
        Loads ld;   // value planes (voff + k) and output adjoints (k, or taps around it)
        for (int t : ex) {
            const Op &o = tape[t];
            const VOp<T> &d = rec[t];
            const int nc = ncontrib(o);
            const size_t at = b.size();   // where this operation's new loads are declared
            b += "        {\n";
            if (o.k == OP_STENCIL && stencils[o.st].mask) {   // a mask is its own transpose
                const Stencil &St = stencils[o.st];
                b += "            const T c0 = wout(x + " + S(St.mx) + ", y + " + S(St.my) + ", nx, ny) ? " +
                     ld.get(A, d.aout, 0, 0, true, "0") + " : T(0);\n";
            } else if (o.k == OP_STENCIL) {   // transpose: gathered from the output adjoint around the node
                const Stencil &St = stencils[o.st];
                b += "            T c0 = T(0);\n";
                std::string plain;
                for (int i = 0; i < St.n; ++i)
                    plain += "            c0 += " + A.c(St.w[i]) + " * " + ld.get(A, d.aout, -St.dx[i], -St.dy[i], true, "0") +
                             ";\n";
                if (walls()) {   // interior nodes: no mirror image lies in the domain
                    b += "            if (inner) {\n" + plain + "            } else {\n";
                    for (int i = 0; i < St.n; ++i)
                        b += "            c0 += " + A.c(St.w[i]) + " * wadj(" + A.p(d.aout) + ", x, y, " + S(-St.dx[i]) +
                             ", " + S(-St.dy[i]) + ", nx, ny, T(" + S(o.sgx) + "), T(" + S(o.sgy) + "));\n";
                    b += "            }\n";
                } else {
                    b += plain;
                }
            } else {
                b += "            T g = " + (d.aout ? ld.get(A, d.aout, 0, 0, false, "0") : std::string("T(0)")) +
                     (d.rout >= 0 ? " + s" + S(d.rout) : std::string("")) + ";\n";
                if (o.k != OP_LIN && o.k != OP_SQRT) b += "            const T a = " + ld.get(A, d.in[0], 0, 0, false, "voff") + ";\n";
                if (o.k == OP_MUL || o.k == OP_DIV) b += "            const T bb = " + ld.get(A, d.in[1], 0, 0, false, "voff") + ";\n";
                if (o.k == OP_SQRT) b += "            const T z = " + ld.get(A, d.out, 0, 0, false, "voff") + ";\n";
                switch (o.k) {
                case OP_LIN:
                    for (int i = 0; i < nc; ++i) b += "            const T c" + S(i) + " = " + A.c((double)d.c[i]) + " * g;\n";
                    break;
                case OP_SCALEP:
                    b += "            const T c0 = " + A.c((double)d.c0) + " * g;\n";
                    b += "            q" + S(o.param) + " += (double)a * (double)g;\n";
                    pgr = true;
                    break;
                case OP_MUL: b += "            const T c0 = bb * g, c1 = a * g;\n"; break;
                case OP_DIV: b += "            const T c0 = g / bb, c1 = -(g * a / (bb * bb));\n"; break;
                case OP_POW3: b += "            const T c0 = T(3) * a * a * g;\n"; break;
                case OP_SQRT: b += "            const T c0 = g / (T(2) * z);\n"; break;
                case OP_CLAMP1: b += "            const T c0 = (a >= T(-1) && a <= T(1)) ? g : T(0);\n"; break;
                default: b += "            const T c0 = -(g / (a * a));\n"; break;   // OP_RECIP
                }
            }
            for (int i = 0; i < nc; ++i) {
                const std::string q = "s" + S(d.rslot[i]);
                b += "            " + q + " = " + (((d.rassign >> i) & 1u) ? "c" + S(i) : q + " + c" + S(i)) + ";\n";
            }
            b += "        }\n";
            b.insert(at, ld.decl);
            ld.decl.clear();
        }
        for (int i = 0; i < G.nfl; ++i) {
            const VFlush<T> &F = hfl[G.fl0 + i];
            const std::string dst = A.p(F.dst);
            b += "        " + dst + "[k] = " + (F.assign ? std::string("") : dst + "[k] + ") + "s" + S(F.slot) + ";\n";
        }
        std::string f = A.decl("KR" + S(gi));
        f += "extern \"C\" __global__ void " + bounds() + " r" + S(gi) + "(const KR" + S(gi) +
             " A, double *pgrad, long long N, long long voff, int nx, int ny)\n{\n"
             "    double q0 = 0.0, q1 = 0.0, q2 = 0.0, q3 = 0.0;\n"
             "    const long long tiles_x = (nx + 31) / 32, tpp = tiles_x * ((ny + JTY - 1) / JTY);\n"
             "    for (long long t = blockIdx.x; t < tpp; t += gridDim.x) {\n"
             "        int x, y;\n"
             "        long long k;\n"
             "        if (!tile_node(t, tiles_x, tpp, nx, ny, N, x, y, k)) continue;\n" + inner_flag();
        for (int q = 0; q < nslots; ++q) f += "        T s" + S(q) + " = T(0);\n";
        f += b + "    }\n";
        if (pgr) f += "    pgrad_add(q0, q1, q2, q3, pgrad);\n";
        return f + "}\n";
    }

    // Source of the wall helpers of a walled tape's kernels (empty when every
    // axis is periodic).  A wall stands halfway beyond the last node: across
    // it a stencil reads the mirror image times the ghost sign, and the
    // transpose of a tap gathers the output adjoint at the tap's offset from
    // the node and from each of its mirror images across the walls (times the
    // same signs), zero wherever that lands outside the domain.
    std::string wall_helpers() const
    {
        if (!walls()) return "";
        return "constexpr int WX = " + S(!perx) + ", WY = " + S(!pery) + ";   // walled axes\n"
            "__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }\n"
            "// (xx, yy) lies across a wall\n"
            "__device__ __forceinline__ bool wout(int xx, int yy, int nx, int ny)\n{\n"
            "    return (WX && (xx < 0 || xx >= nx)) || (WY && (yy < 0 || yy >= ny));\n}\n"
            "// p at (x + dx, y + dy), mirrored across walls with signs sx, sy\n"
            "__device__ __forceinline__ T wtap(const T *p, int x, int y, int dx, int dy, int nx, int ny, T sx, T sy)\n{\n"
            "    int xx = x + dx, yy = y + dy;\n"
            "    T f = T(1);\n"
            "    if (WX) { if (xx < 0) { xx = -1 - xx; f = sx; } else if (xx >= nx) { xx = 2 * nx - 1 - xx; f = sx; } }\n"
            "    else xx = wrapi(xx, nx);\n"
            "    if (WY) { if (yy < 0) { yy = -1 - yy; f *= sy; } else if (yy >= ny) { yy = 2 * ny - 1 - yy; f *= sy; } }\n"
            "    else yy = wrapi(yy, ny);\n"
            "    return f == T(0) ? T(0) : f * __ldg(p + (long long)yy * nx + xx);\n}\n"
            "// p at (xx, yy), zero across a wall\n"
            "__device__ __forceinline__ T wext(const T *p, int xx, int yy, int nx, int ny)\n{\n"
            "    if (wout(xx, yy, nx, ny)) return T(0);\n"
            "    return __ldg(p + (long long)wrapi(yy, ny) * nx + wrapi(xx, nx));\n}\n"
            "// transpose of a tap at (dx, dy) = minus the stencil's offset\n"
            "__device__ __forceinline__ T wadj(const T *p, int x, int y, int dx, int dy, int nx, int ny, T sx, T sy)\n{\n"
            "    T acc = wext(p, x + dx, y + dy, nx, ny);\n"
            "    const int xl = -1 - x + dx, xh = 2 * nx - 1 - x + dx, yl = -1 - y + dy, yh = 2 * ny - 1 - y + dy;\n"
            "    if (WY && sy != T(0)) acc += sy * (wext(p, x + dx, yl, nx, ny) + wext(p, x + dx, yh, nx, ny));\n"
            "    if (WX && sx != T(0)) {\n"
            "        acc += sx * (wext(p, xl, y + dy, nx, ny) + wext(p, xh, y + dy, nx, ny));\n"
            "        if (WY && sy != T(0))\n"
            "            acc += sx * sy * (wext(p, xl, yl, nx, ny) + wext(p, xl, yh, nx, ny) + wext(p, xh, yl, nx, ny) +\n"
            "                              wext(p, xh, yh, nx, ny));\n"
            "    }\n"
            "    return acc;\n}\n";
    }

    // Declaration of `inner` in a walled tape's kernels: the node lies at
    // least the stencils' reach from every wall, so every tap of a stencil
    // lands inside the domain and no mirror image of a transposed tap does
    // (wtap and wadj reduce there to the plain tap, bit for bit).
    std::string inner_flag() const
    {
        if (!walls()) return "";
        int rx = 0, ry = 0;
        for (const Stencil &St : stencils)
            for (int i = 0; i < St.n; ++i) {
                rx = std::max(rx, std::abs(St.dx[i]));
                ry = std::max(ry, std::abs(St.dy[i]));
            }
        return "        const bool inner = (!WX || (x >= " + S(rx) + " && x < nx - " + S(rx) + ")) && (!WY || (y >= " +
               S(ry) + " && y < ny - " + S(ry) + "));\n";
    }

    // Write the schedule out as compiled level kernels (unless switched off
    // by LBM_ADJOINT_COMPILED=0); jit says whether they run this tape.
    void compile_levels(const std::vector<VOp<T>> &rec, const std::vector<std::vector<int>> &rex)
    {
        jit = false;
        jfwd.assign(fgroups.size(), JKernel{});
        jrev.assign(rgroups.size(), JKernel{});
        pingpong = false;
        const char *sw = getenv("LBM_ADJOINT_COMPILED");
        if (sw && sw[0] == '0') return;
        static_assert(NPARAM == 4, "generated kernels sum four parameter gradients");
        std::string src = std::string("typedef ") + (sizeof(T) == 8 ? "double" : "float") + " T;\n" +
            "constexpr int JTY = " + S(JTY) + ";\n" +
            "__device__ __forceinline__ long long nbi(int x, int y, int dx, int dy, int nx, int ny)\n{\n"
            "    int xx = x + dx, yy = y + dy;\n"
            "    xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);\n"
            "    yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);\n"
            "    return (long long)yy * nx + xx;\n}\n" + wall_helpers() +
            "// Node of this thread in tile t of a batch: tiles of 32 x JTY nodes (a warp per\n"
            "// row, so vertical stencil taps are mostly shared through L1), tiles_x per\n"
            "// row of tiles, tpp per step; false outside the grid.\n"
            "__device__ __forceinline__ bool tile_node(long long t, long long tiles_x, long long tpp, int nx, int ny,\n"
            "                                          long long N, int &x, int &y, long long &k)\n{\n"
            "    const long long b = t / tpp, r = t - b * tpp, ty = r / tiles_x;\n"
            "    x = (int)(r - ty * tiles_x) * 32 + (int)(threadIdx.x & 31);\n"
            "    y = (int)ty * JTY + (int)(threadIdx.x >> 5);\n"
            "    k = b * N + (long long)y * nx + x;\n"
            "    return x < nx && y < ny;\n}\n"
            "__device__ __forceinline__ void pgrad_add(double q0, double q1, double q2, double q3, double *pg)\n{\n"
            "    __shared__ double red[4][32];\n"
            "    double v[4] = {q0, q1, q2, q3};\n"
            "    for (int q = 0; q < 4; ++q) {\n"
            "        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);\n"
            "        if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v[q];\n"
            "    }\n"
            "    __syncthreads();\n"
            "    if (threadIdx.x < 4) {\n"
            "        double t = 0.0;\n"
            "        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];\n"
            "        if (t != 0.0) atomicAdd(pg + threadIdx.x, t);\n"
            "    }\n}\n";
        std::vector<ArgPack> af(fgroups.size()), ar(rgroups.size());
        for (size_t g = 0; g < fgroups.size(); ++g) src += gen_fwd((int)g, af[g]);
        for (size_t g = 0; g < rgroups.size(); ++g) {
            int nslots = 0;   // accumulation slots: every slot a record or flush names
            for (int t : rex[g]) {
                const VOp<T> &d = rec[t];
                for (int i = 0; i < ncontrib(tape[t]); ++i) nslots = std::max(nslots, d.rslot[i] + 1);
                nslots = std::max(nslots, d.rout + 1);
            }
            for (int i = 0; i < rgroups[g].nfl; ++i) nslots = std::max(nslots, hfl[rgroups[g].fl0 + i].slot + 1);
            src += gen_rev((int)g, rex[g], rec, nslots, ar[g]);
        }
        cudaLibrary_t lib = lbm_jit::library(src);
        if (!lib) {
            static bool told = false;
            if (!told) fprintf(stderr, "lbm adjoint: compiled level kernels unavailable (%s); interpreting the tape\n",
                               lbm_jit::reason().c_str());
            told = true;
            return;
        }
        for (size_t g = 0; g < fgroups.size(); ++g) {
            if (cudaLibraryGetKernel(&jfwd[g].k, lib, ("f" + S((int)g)).c_str()) != cudaSuccess) { cudaGetLastError(); return; }
            jfwd[g].pack = af[g].pack();
        }
        for (size_t g = 0; g < rgroups.size(); ++g) {
            if (cudaLibraryGetKernel(&jrev[g].k, lib, ("r" + S((int)g)).c_str()) != cudaSuccess) { cudaGetLastError(); return; }
            jrev[g].pack = ar[g].pack();
            jrev[g].np = (int)ar[g].ptr.size();
        }
        jit = true;
    }

    // Reverse records of one kernel: the live operations ex (execution
    // order) split into phases of at most STAGE staged loads (a stencil with
    // more taps gets a phase of its own); phase p stages into buffer p % 2 of
    // Sb slots after the kernel's `base` accumulation slots.
    void add_rgroup(const std::vector<int> &ex, int base, const std::vector<VOp<T>> &rec)
    {
        struct Load { const T *p; int dx, dy, val; };
        std::vector<std::vector<Load>> loads(ex.size());
        for (size_t j = 0; j < ex.size(); ++j) {
            const Op &o = tape[ex[j]];
            const VOp<T> &d = rec[ex[j]];
            auto &L = loads[j];
            if (o.k == OP_STENCIL) {
                const Stencil &S = stencils[o.st];
                for (int i = 0; i < S.n; ++i) L.push_back({d.aout, -S.dx[i], -S.dy[i], 0});
            } else {
                if (o.k != OP_LIN && o.k != OP_SQRT) L.push_back({d.in[0], 0, 0, 1});
                if (o.k == OP_MUL || o.k == OP_DIV) L.push_back({d.in[1], 0, 0, 1});
                if (o.k == OP_SQRT) L.push_back({d.out, 0, 0, 1});
                if (d.aout) L.push_back({d.aout, 0, 0, 0});
            }
        }
        // phase boundaries
        std::vector<std::pair<int, int>> ranges;   // [first op, end op)
        int sb = 0;
        for (size_t j = 0, first = 0, cnt = 0; j <= ex.size(); ++j) {
            const size_t need = j < ex.size() ? loads[j].size() : 0;
            if (j == ex.size() || (cnt + need > (size_t)STAGE && j > first)) {
                if (j > first) {
                    ranges.push_back({(int)first, (int)j});
                    sb = std::max(sb, (int)cnt);
                }
                first = j;
                cnt = 0;
            }
            cnt += need;
        }
        RGroup G{};
        G.op0 = (int)hrop.size();
        G.pre0 = (int)hpre.size();
        G.ph0 = (int)hph.size();
        G.nph = (int)ranges.size();
        G.slots = base + sb * std::min(2, G.nph);
        for (int p = 0; p < G.nph; ++p) {
            VPhase P{ranges[p].first, ranges[p].second - ranges[p].first, (int)hpre.size() - G.pre0, 0};
            int cnt = 0;
            auto stage = [&](const Load &ld) {
                const int s = base + (p % 2) * sb + cnt++;
                hpre.push_back({ld.p, (short)s, (signed char)ld.dx, (signed char)ld.dy, ld.val});
                return s;
            };
            for (int j = ranges[p].first; j < ranges[p].second; ++j) {
                const Op &o = tape[ex[j]];
                const VOp<T> &d = rec[ex[j]];
                VRop<T> r{};
                r.k = o.k;
                r.nc = ncontrib(o);
                r.param = o.param;
                r.st = o.st;
                r.rassign = d.rassign;
                for (int i = 0; i < MAXIN; ++i) { r.rslot[i] = d.rslot[i]; r.c[i] = d.c[i]; }
                r.rout = d.rout;
                r.c0 = d.c0;
                r.sa = r.sb = r.sz = r.sg = r.stap = -1;
                const auto &L = loads[j];
                if (o.k == OP_STENCIL) {
                    r.stap = (short)(base + (p % 2) * sb + cnt);
                    for (const Load &ld : L) stage(ld);
                } else {
                    size_t i = 0;
                    if (o.k != OP_LIN && o.k != OP_SQRT) r.sa = (short)stage(L[i++]);
                    if (o.k == OP_MUL || o.k == OP_DIV) r.sb = (short)stage(L[i++]);
                    if (o.k == OP_SQRT) r.sz = (short)stage(L[i++]);
                    if (d.aout) r.sg = (short)stage(L[i++]);
                }
                hrop.push_back(r);
            }
            P.ne = cnt;
            hph.push_back(P);
        }
        G.nops = (int)hrop.size() - G.op0;
        G.npre = (int)hpre.size() - G.pre0;
        rgroups.push_back(G);
    }

    void upload()
    {
        check(cudaStreamSynchronize(st));   // earlier kernels may still read the old records
        if (rst && rst != st) check(cudaStreamSynchronize(rst));
        if (!d_tab) {
            std::vector<DStencil> tab(stencils.size());
            for (size_t i = 0; i < stencils.size(); ++i) {
                tab[i].n = stencils[i].n;
                for (int j = 0; j < stencils[i].n; ++j) {
                    tab[i].dx[j] = stencils[i].dx[j];
                    tab[i].dy[j] = stencils[i].dy[j];
                    tab[i].w[j] = stencils[i].w[j];
                }
            }
            check(cudaMalloc((void **)&d_tab, sizeof(DStencil) * tab.size()));
            if (err == cudaSuccess)
                check(cudaMemcpy(d_tab, tab.data(), sizeof(DStencil) * tab.size(), cudaMemcpyHostToDevice));
            std::vector<DW<T>> tw(stencils.size());
            for (size_t i = 0; i < stencils.size(); ++i) {
                tw[i] = DW<T>{};
                tw[i].n = stencils[i].n;
                for (int j = 0; j < stencils[i].n; ++j) tw[i].w[j] = (T)stencils[i].w[j];
            }
            check(cudaMalloc((void **)&d_tw, sizeof(DW<T>) * tw.size()));
            if (err == cudaSuccess)
                check(cudaMemcpy(d_tw, tw.data(), sizeof(DW<T>) * tw.size(), cudaMemcpyHostToDevice));
        }
        auto put_array = [&](auto &h, auto *&d, size_t &cap) {
            using E = typename std::remove_reference<decltype(h)>::type::value_type;
            if (h.size() > cap) {
                if (d) cudaFree(d);
                cap = h.size();
                check(cudaMalloc((void **)&d, sizeof(E) * cap));
            }
            if (err == cudaSuccess && !h.empty())
                check(cudaMemcpy(d, h.data(), sizeof(E) * h.size(), cudaMemcpyHostToDevice));
        };
        put_array(hfwd, d_fwd, cap_fwd);
        put_array(hrop, d_rop, cap_rop);
        put_array(hpre, d_pre, cap_pre);
        put_array(hph, d_ph, cap_ph);
        put_array(hfl, d_fl, cap_fl);
    }

    // Forward pass of the tape for steps lo .. lo + cnt - 1 (cnt <= Bcap) in
    // one batch on st: leaf i of step j is read at its recorded source plus
    // j * leaf_stride; the step's values land at (j - lo) N in value buffer vb.
    // With leaves_in_place the leaf values are already in value buffer vb.
    void forward(int lo, int cnt, int vb = 0, bool leaves_in_place = false)
    {
        for (size_t b = 0; !leaves_in_place && b < leaves.size(); b += MAXLEAF) {
            Leaves<T> Lv{};
            Lv.n = (int)std::min<size_t>(MAXLEAF, leaves.size() - b);
            for (int i = 0; i < Lv.n; ++i) {
                Lv.dst[i] = val[leaves[b + i].first] + vbase(vb);
                const size_t esz = leaf_f32[b + i] ? sizeof(float) : sizeof(T);
                Lv.src[i] = (const char *)leaves[b + i].second + esz * (size_t)(leaf_stride * lo);
                if (leaf_f32[b + i]) Lv.f32 |= 1u << i;
            }
            kk_leaves<T><<<std::max(1, std::min(nb * cnt, 65535)), NTH, 0, st>>>(Lv, N, cnt, leaf_stride);
        }
        const int nblk = (int)std::min<long long>((N * cnt + NTV - 1) / NTV, 65535);
        if (jit) {
            long long Nn = N, Ntot = N * cnt, voff = vbase(vb);
            int nxx = nx, nyy = ny;
            for (JKernel &J : jfwd) {
                void *args[] = {J.pack.data(), &Nn, &Ntot, &voff, &nxx, &nyy};
                check(cudaLaunchKernel((const void *)J.k, dim3(std::max(1, (int)std::min<long long>((Ntot + JT - 1) / JT, 65535))),
                                       dim3(JT), args, 0, st));
            }
        } else {
            for (const Group &G : fgroups)
                kk_vm_fwd<T><<<nblk, NTV, VmLayout<T>::bytes(ntab, G.n, G.slots), st>>>(
                    d_tab, ntab, d_fwd + G.off, G.n, nx, ny, N, N * cnt, vbase(vb));
        }
        check(cudaGetLastError());
    }

    // Let consecutive reverse passes of a step tape hand the state adjoint
    // over without copies: a second argument pack of each compiled reverse
    // kernel has the adjoint planes of the output state (the seeds, out[i])
    // and of the input state (the leaves, in[i]) exchanged.  A pass with
    // pack v reads its seeds from one set and leaves the input state's
    // adjoint in the other, where the next pass, with pack 1 - v, finds its
    // seeds.  Needs distinct, disjoint output and input planes, seeded by
    // assignment, and every leaf reached by the sweep (so the leaf planes
    // are overwritten, not added to, by each pass); false otherwise.
    bool enable_pingpong(const int *in, const int *out, int n)
    {
        pingpong = false;
        if (!jit || (int)seeds.size() != n) return false;
        std::map<const void *, const void *> sw;
        for (int i = 0; i < n; ++i) {
            if (seeds[i].first != out[i] || seed_add[i] || !flowed[in[i]] || !adj[in[i]] || !adj[out[i]]) return false;
            if (!sw.emplace(adj[out[i]], adj[in[i]]).second || !sw.emplace(adj[in[i]], adj[out[i]]).second) return false;
        }
        for (JKernel &J : jrev) {
            J.pack_sw = J.pack;
            for (int i = 0; i < J.np; ++i) {
                auto it = sw.find((const void *)(uintptr_t)J.pack[i]);
                if (it != sw.end()) J.pack_sw[i] = (unsigned long long)(uintptr_t)it->second;
            }
        }
        pingpong = true;
        return true;
    }

    // Reverse pass, on rst, of step b of value buffer vb (values at b N in
    // it).  ver < 0: the seeded adjoints start from the seeds; ver 0 / 1
    // (compiled kernels with ping-pong): argument pack ver, seeded first
    // only when seed is set.
    void reverse(int b, int vb = 0, int ver = -1, bool seed = true)
    {
        cudaStream_t s = rst ? rst : st;
        for (size_t s0 = 0; seed && s0 < seeds.size(); s0 += MAXLEAF) {
            Leaves<T> Lv{};
            Lv.n = (int)std::min<size_t>(MAXLEAF, seeds.size() - s0);
            for (int i = 0; i < Lv.n; ++i) {
                Lv.dst[i] = adj[seeds[s0 + i].first];
                Lv.src[i] = seeds[s0 + i].second;
                if (seed_add[s0 + i]) Lv.add |= 1u << i;
            }
            kk_leaves<T><<<nb, NTH, 0, s>>>(Lv, N, 1, 0);
        }
        if (jit) {
            long long Nn = N, voff = vbase(vb) + (long long)b * N;
            int nxx = nx, nyy = ny;
            double *pg = d_pgrad;
            for (JKernel &J : jrev) {
                void *args[] = {(ver == 1 ? J.pack_sw : J.pack).data(), &pg, &Nn, &voff, &nxx, &nyy};
                check(cudaLaunchKernel((const void *)J.k, dim3(std::max(1, (int)std::min<long long>((Nn + JT - 1) / JT, 8192))),
                                       dim3(JT), args, 0, s));
            }
        } else {
            for (const RGroup &G : rgroups) {
                const RevArgs<T> A{d_tw, d_rop + G.op0, d_pre + G.pre0, d_ph + G.ph0, d_fl + G.fl0,
                                   ntab, G.nops, G.npre, G.nph, G.nfl};
                kk_vm_rev<T><<<nbv, NTV, RevLayout<T>::bytes(ntab, G.nops, G.npre, G.nph, G.nfl, G.slots), s>>>(
                    A, d_pgrad, nx, ny, N, vbase(vb) + (long long)b * N);
            }
        }
        check(cudaGetLastError());
    }

    // dst[i] = adjoint of plane ids[i] (zero where none flowed), on rst.
    void collect(const int *ids, T *const *dst, int n)
    {
        cudaStream_t s = rst ? rst : st;
        for (int b = 0; b < n; b += MAXLEAF) {
            Leaves<T> Lv{};
            Lv.n = std::min(MAXLEAF, n - b);
            for (int i = 0; i < Lv.n; ++i) {
                const bool f = ids[b + i] < (int)flowed.size() && flowed[ids[b + i]];
                Lv.dst[i] = dst[b + i];
                Lv.src[i] = f ? adj[ids[b + i]] : nullptr;
                if (!f) Lv.zero |= 1u << i;
            }
            kk_leaves<T><<<nb, NTH, 0, s>>>(Lv, N, 1, 0);
        }
        check(cudaGetLastError());
    }
};

// Stencil table indices.
enum { S_GX, S_GY, S_LAP, S_D1X, S_D1Y, S_D2X, S_D2Y, S_FILTER, S_SHIFT0, S_BB0 = S_SHIFT0 + 9 };
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
    std::vector<Stencil> S(S_BB0 + 9);
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
    for (int q = 0; q < 9; ++q) {   // halfway bounce-back: f_q(x) = f*_opp(q)(x) where x - c_q is across a wall
        add(S[S_BB0 + q], 0, 0, 1.0);
        S[S_BB0 + q].mask = true;
        S[S_BB0 + q].mx = -CX[q];
        S[S_BB0 + q].my = -CY[q];
    }
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

    // isotropic gradient of a plane whose parities across walls are (sx, sy)
    int gx(int a, int sx = 1, int sy = 1) { return E.sten(a, S_GX, sx, sy); }
    int gy(int a, int sx = 1, int sy = 1) { return E.sten(a, S_GY, sx, sy); }

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
        // F_s = kappa div(|grad phi|^2 I - grad phi grad phi); the product of the
        // components of grad phi is odd across walls on either axis
        F.Fsx = E.scalep(E.lin({{gx(gy2), 1.0}, {gy(gxy, -1, -1), -1.0}}), P_KAPPA);
        F.Fsy = E.scalep(E.lin({{gx(gxy, -1, -1), -1.0}, {gy(gx2), 1.0}}), P_KAPPA);
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
        du[0] = gx(ux, -1, -1); du[1] = gy(ux, -1, -1); du[2] = gx(uy, -1, -1); du[3] = gy(uy, -1, -1);   // no slip
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
        // J_x is odd across an x wall and even across a y wall, J_y the reverse
        return E.lin({{E.sten(jx, S_D1X, -1, 1), 1.0}, {E.sten(jy, S_D1Y, 1, -1), 1.0}});
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
            if (E.walls()) {   // pulls from across a wall take the node's opposite population
                int qo = 0;
                while (CX[qo] != -CX[q] || CY[qo] != -CY[q]) ++qo;
                o.f[q] = E.lin({{E.sten(fs[q], S_SHIFT0 + q, 0, 0), 1.0}, {E.sten(fs[qo], S_BB0 + q), 1.0}});
                o.g[q] = E.lin({{E.sten(gs[q], S_SHIFT0 + q, 0, 0), 1.0}, {E.sten(gs[qo], S_BB0 + q), 1.0}});
            } else {
                o.f[q] = E.sten(fs[q], S_SHIFT0 + q);
                o.g[q] = E.sten(gs[q], S_SHIFT0 + q);
            }
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
        o.ux = E.sten(ukx, S_FILTER, -1, -1);
        o.uy = E.sten(uky, S_FILTER, -1, -1);
        o.uhx = ukx; o.uhy = uky;
        o.upx = E.lin({{s.ux, 1.0}});   // u^{n-1} of the next step, a plane of its own
        o.upy = E.lin({{s.uy, 1.0}});
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
    std::vector<void *> seg;       // one segment of states (when a segment spans several batches)
    void *init4 = nullptr;         // phi0, p0, ux0, uy0
    void *final_state = nullptr;   // state after nsteps
    void *lam = nullptr;           // adjoint state, NSTATE planes
    void *eng = nullptr;           // Engine<T> of the handle's arithmetic type
    bool eng64 = false;            // eng is an Engine<double>
    bool ready = false;
    cudaStream_t rs = nullptr;     // reverse-pass stream (high priority, non-blocking)
    int engine = -1;               // last reverse sweep: 1 compiled level kernels, 0 interpreter
    cudaEvent_t ev[5]{};           // batch forward done (2), batch reverse done (2), sweep done
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
    void *r[8] = {phi_cur(h), h->pf, h->ux[h->ucur], h->uy[h->ucur], h->uhx, h->uhy, h->ux[1 - h->ucur], h->uy[1 - h->ucur]};
    return r[i - 18];
}

// The 26 state planes to (out) or from a packed buffer, one launch on the
// handle's stream.
template <typename T> cudaError_t copy_state_t(lbm_handle *h, void *buf, bool out)
{
    Leaves<T> Lv{};
    Lv.n = NSTATE;
    for (int i = 0; i < NSTATE; ++i) {
        T *packed = (T *)buf + (size_t)i * h->N;
        Lv.dst[i] = out ? packed : (T *)state_ptr(h, i);
        Lv.src[i] = out ? state_ptr(h, i) : packed;
    }
    kk_leaves<T><<<blocks_for(h->N), NTH, 0, h->stream>>>(Lv, h->N, 1, 0);
    return cudaGetLastError();
}
cudaError_t copy_state_out(lbm_handle *h, void *dst)
{
    return h->elem == sizeof(double) ? copy_state_t<double>(h, dst, true) : copy_state_t<float>(h, dst, true);
}
// The 26 state planes to 26 separate planes, one launch on the handle's stream.
template <typename T> cudaError_t copy_state_to(lbm_handle *h, T *const *dst)
{
    Leaves<T> Lv{};
    Lv.n = NSTATE;
    for (int i = 0; i < NSTATE; ++i) {
        Lv.dst[i] = dst[i];
        Lv.src[i] = state_ptr(h, i);
    }
    kk_leaves<T><<<blocks_for(h->N), NTH, 0, h->stream>>>(Lv, h->N, 1, 0);
    return cudaGetLastError();
}
// The checkpoints hold phi_hi only: a restored FP32 state starts with
// phi_lo = 0, so regeneration follows the forward run to within the rounding
// of phi (the sweep itself reads phi_hi).
cudaError_t copy_state_in(lbm_handle *h, const void *src)
{
    void *s = const_cast<void *>(src);
    if (h->elem == sizeof(double)) return copy_state_t<double>(h, s, false);
    cudaError_t e = cudaMemsetAsync(h->philo, 0, sizeof(float) * (size_t)h->N, h->stream);
    return e != cudaSuccess ? e : copy_state_t<float>(h, s, false);
}

// The reverse sweep runs in the handle's arithmetic type T (the adjoint
// state too); only the parameter gradients are summed in FP64.
template <typename T> lbm_status run_reverse(lbm_handle *h, const double *seed, double *dphi0, double *dsigma, double *dM)
{
    using D = T;
    lbm_adjoint *A = h->adj;
    const size_t n = (size_t)h->N, pb = sizeof(T) * n, pd = sizeof(D) * n;
    Engine<D> *E = (Engine<D> *)A->eng;
    if (!E) {
        E = new Engine<D>();
        A->eng = E;
        A->eng64 = sizeof(D) == sizeof(double);
    }
    E->nx = h->grid.nx; E->ny = h->grid.ny; E->N = h->N; E->st = h->stream; E->nb = blocks_for(h->N);
    E->perx = h->grid.periodic_x ? 1 : 0;
    E->pery = h->grid.periodic_y ? 1 : 0;
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
    std::vector<D> seed_t(seed, seed + n);
    cudaMemcpyAsync(lam + 18 * n, seed_t.data(), pd, cudaMemcpyHostToDevice, h->stream);
    cudaStreamSynchronize(h->stream);
    Recorder<D> R(*E, P);
    const int nseg = (A->nsteps + A->every - 1) / A->every;
    // the step's tape, recorded once: leaf i reads slot i of a stored state,
    // and a segment's states sit NSTATE planes apart
    E->reset();
    StateIds in;
    // leaf i is slot i of a stored state; its source is set below when the
    // segment buffer is used
    for (int i = 0; i < NSTATE; ++i) *slot(in, i) = E->leaf((const T *)nullptr);
    StateIds out = R.step(in);
    for (int i = 0; i < NSTATE; ++i) E->seed(*slot(out, i), lam + i * n);
    E->Bwant = A->every;
    if (const char *cap = getenv("LBM_ADJOINT_BATCH"))   // at most this many steps per batch
        E->Bwant = std::max(1, std::min(A->every, atoi(cap)));
    E->leaf_stride = (long long)NSTATE * (long long)n;
    E->prepare();
    if (E->err != cudaSuccess) return afail(h, LBM_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(E->err));
    if (E->walls() && !E->jit)   // the tape interpreter's stencils are periodic only
        return afail(h, LBM_ERR_ARG, "adjoint: walls need the compiled level kernels" +
                                         (lbm_jit::reason().empty() ? std::string() : " (" + lbm_jit::reason() + ")"));
    const int Bc = std::max(1, std::min(E->Bcap, E->Bwant)), nvb = E->nvbuf;
    int ids[NSTATE], ido[NSTATE];
    D *dst[NSTATE];
    for (int i = 0; i < NSTATE; ++i) {
        ids[i] = *slot(in, i);
        ido[i] = *slot(out, i);
        dst[i] = lam + i * n;
    }
    // compiled kernels: consecutive passes hand the state adjoint over by
    // exchanging argument packs instead of collecting and re-seeding it
    const bool pp = E->enable_pingpong(ids, ido, NSTATE);
    int passes = 0;
    // Batches from the last step backwards: each segment from its end, Bc
    // steps at a time.  Producing a batch (regenerating its segment's states
    // with the fused forward kernels when it is the segment's last batch,
    // then the tape's forward pass of the batch at once) runs on the handle's
    // stream; its reverse pass, step by step, on the reverse stream.  With two
    // value buffers the next batch is produced while this one is reversed.
    struct Batch { int seg, lo, hi; bool first; };
    std::vector<Batch> bl;
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
        const int len = std::min(A->every, A->nsteps - sgi * A->every);
        for (int hi = len; hi > 0; hi -= Bc) bl.push_back({sgi, std::max(0, hi - Bc), hi, hi == len});
    }
    if (!A->rs) {
        int lo_pri = 0, hi_pri = 0;
        cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);
        if (cudaStreamCreateWithPriority(&A->rs, cudaStreamNonBlocking, hi_pri) != cudaSuccess)
            return afail(h, LBM_ERR_CUDA, "adjoint: reverse stream");
        for (cudaEvent_t &e : A->ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                return afail(h, LBM_ERR_CUDA, "adjoint: events");
    }
    cudaEvent_t *evF = A->ev, *evR = A->ev + 2;
    E->rst = A->rs;
    // When a batch holds a whole segment, regeneration stores each state
    // straight into the batch's leaf value planes: no segment buffer and no
    // copy of the leaves before the tape's forward pass.
    const bool direct = Bc >= A->every;
    if (!direct) {
        if (!A->seg[0] && cudaMalloc(&A->seg[0], sizeof(T) * n * NSTATE * (size_t)A->every) != cudaSuccess) {
            cudaGetLastError();
            return afail(h, LBM_ERR_OOM, "adjoint: segment buffer");
        }
        for (int i = 0; i < NSTATE; ++i) E->leaves[i].second = (const T *)A->seg[0] + i * n;
    }
    auto produce = [&](int c) -> lbm_status {
        const Batch &b = bl[c];
        const int vb = c % nvb;
        if (direct && c >= nvb) cudaStreamWaitEvent(h->stream, evR[vb], 0);   // the buffer's last reader
        if (b.first) {
            if (copy_state_in(h, A->ckpt[b.seg]) != cudaSuccess) return afail(h, LBM_ERR_CUDA, "adjoint: restore");
            const int len = b.hi;
            for (int j = 0; j < len; ++j) {
                cudaError_t e;
                if (direct) {
                    D *to[NSTATE];
                    for (int i = 0; i < NSTATE; ++i) to[i] = E->leaf_dst(i, vb, j);
                    e = copy_state_to<D>(h, to);
                } else {
                    e = copy_state_out(h, (char *)A->seg[0] + (size_t)j * NSTATE * pb);
                }
                if (e != cudaSuccess) return afail(h, LBM_ERR_CUDA, "adjoint: segment store");
                if (j + 1 < len) {
                    lbm_status st = lbm_internal_step(h);
                    if (st) return st;
                }
            }
        }
        if (!direct && c >= nvb) cudaStreamWaitEvent(h->stream, evR[vb], 0);   // the buffer's last reader
        E->forward(b.lo, b.hi - b.lo, vb, direct);
        cudaEventRecord(evF[vb], h->stream);
        return LBM_OK;
    };
    auto consume = [&](int c) {
        const Batch &b = bl[c];
        const int vb = c % nvb;
        cudaStreamWaitEvent(A->rs, evF[vb], 0);
        for (int j = b.hi - 1; j >= b.lo; --j, ++passes) {
            if (pp) {
                E->reverse(j - b.lo, vb, passes % 2, passes == 0);
            } else {
                E->reverse(j - b.lo, vb);
                E->collect(ids, dst, NSTATE);
            }
        }
        cudaEventRecord(evR[vb], A->rs);
    };
    lbm_status pst = LBM_OK;
    for (int c = 0; c < nvb - 1 && c < (int)bl.size() && !pst; ++c) pst = produce(c);
    for (int c = 0; c < (int)bl.size() && !pst; ++c) {
        if (c + nvb - 1 < (int)bl.size()) pst = produce(c + nvb - 1);
        if (!pst) consume(c);
        if (!pst && E->err != cudaSuccess)
            pst = afail(h, LBM_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(E->err));
    }
    const bool step_jit = E->jit;
    // the last pass left the input state's adjoint in the planes of pack (passes - 1) % 2
    if (!pst && pp && passes > 0) E->collect((passes - 1) % 2 == 0 ? ids : ido, dst, NSTATE);
    // join: the handle's stream waits for the reverse stream's work
    cudaEventRecord(A->ev[4], A->rs);
    cudaStreamWaitEvent(h->stream, A->ev[4], 0);
    E->rst = nullptr;
    if (pst) {
        cudaStreamSynchronize(h->stream);
        return pst;
    }
    // through the initialisation from (phi0, p0, u0)
    E->reset();
    const T *i4 = (const T *)A->init4;
    int phi0 = E->leaf(i4), p0 = E->leaf(i4 + n), ux0 = E->leaf(i4 + 2 * n), uy0 = E->leaf(i4 + 3 * n);
    StateIds s0 = R.init(phi0, p0, ux0, uy0);
    for (int i = 0; i < NSTATE; ++i) E->seed(*slot(s0, i), lam + i * n);
    E->run();
    A->engine = step_jit && E->jit ? 1 : 0;
    std::vector<D> g(n, D(0));
    if (E->flowed[phi0]) cudaMemcpyAsync(g.data(), E->adj[phi0], pd, cudaMemcpyDeviceToHost, h->stream);
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
    if (A->rs) cudaStreamSynchronize(A->rs);
    for (cudaEvent_t e : A->ev) if (e) cudaEventDestroy(e);
    if (A->rs) cudaStreamDestroy(A->rs);
    cudaFree(A->init4);
    cudaFree(A->final_state);
    cudaFree(A->lam);
    if (A->eng && A->eng64) {
        auto *E = (Engine<double> *)A->eng;
        E->release_all();
        delete E;
    } else if (A->eng) {
        auto *E = (Engine<float> *)A->eng;
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
    A->seg.assign(1, nullptr);   // allocated by the reverse sweep if a segment spans several batches
    if (!ok) {
        cudaGetLastError();
        lbm_internal_adjoint_free(h);
        return afail(h, LBM_ERR_OOM, "adjoint: checkpoint allocation");
    }
    // the initial fields: phi0, p0, u0 of the fresh state
    cudaMemcpyAsync(A->init4, phi_cur(h), pb, cudaMemcpyDeviceToDevice, h->stream);
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
    lbm_status pst = lbm_internal_poll_device_error(h);
    if (pst) return pst;
    A->ready = true;
    return LBM_OK;
}

int lbm_adjoint_engine(const lbm_handle *h)
{
    return h && h->adj ? h->adj->engine : -1;
}

lbm_status lbm_adjoint_end(lbm_handle *h, const double *dL_dphi, double *dL_dphi0, double *dL_dsigma,
                           double *dL_dM)
{
    if (!h) return LBM_ERR_ARG;
    if (!h->adj || !h->adj->ready) return afail(h, LBM_ERR_STATE, "lbm_adjoint_end needs lbm_adjoint_begin first");
    if (!dL_dphi) return afail(h, LBM_ERR_ARG, "dL_dphi must be non-NULL");
    lbm_status st = h->grid.precision == LBM_FP64 ? run_reverse<double>(h, dL_dphi, dL_dphi0, dL_dsigma, dL_dM)
                                                  : run_reverse<float>(h, dL_dphi, dL_dphi0, dL_dsigma, dL_dM);
    return st ? st : lbm_internal_poll_device_error(h);
}

}  // extern "C"
