// Host-side checks of the adjoint engine's schedule, without a GPU.
//
// lbm_adjoint.cu is compiled with the few CUDA runtime calls the scheduler
// makes replaced by stand-ins (memory queries and allocations succeed with
// host addresses that are never dereferenced; copies and attribute calls do
// nothing; a loaded library is a dummy handle).  For each tape structure the
// step's tape is recorded and scheduled in FP32 and FP64, and the device
// form is checked: every slot index inside its kernel's slot count, every
// global read from a plane that has storage, every staged operand and
// stencil tap loaded in the phase that uses it, no accumulation slot shared
// with a staging slot, every flush in range, the leaves stored.  When
// NVRTC can be opened the generated level kernels are compiled for real,
// and the exchange of argument packs must be possible for the step tape.
// Prints one line per case and exits non-zero on the first failing case.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>

static cudaError_t fake_meminfo(size_t *f, size_t *t)
{
    *f = 200ull << 30;
    *t = 280ull << 30;
    return cudaSuccess;
}
// Distinct, non-overlapping addresses that are never dereferenced.
static cudaError_t fake_malloc(void **p, size_t bytes)
{
    static uintptr_t next = uintptr_t(1) << 40;
    *p = (void *)next;
    next += (bytes + 4095) / 4096 * 4096 + 4096;
    return cudaSuccess;
}
template <typename A, typename B> static cudaError_t fake_memcpy(A, B, size_t, cudaMemcpyKind) { return cudaSuccess; }
static cudaError_t fake_sync(cudaStream_t) { return cudaSuccess; }
template <typename F> static cudaError_t fake_attr(F, cudaFuncAttribute, int) { return cudaSuccess; }
static cudaError_t fake_getdev(int *d)
{
    *d = 0;
    return cudaSuccess;
}
static cudaError_t fake_libload(cudaLibrary_t *l, const void *, cudaJitOption *, void **, unsigned, cudaLibraryOption *,
                                void **, unsigned)
{
    *l = (cudaLibrary_t)0x1;
    return cudaSuccess;
}
static cudaError_t fake_libkernel(cudaKernel_t *k, cudaLibrary_t, const char *)
{
    *k = (cudaKernel_t)0x1;
    return cudaSuccess;
}
#define cudaMemGetInfo fake_meminfo
#define cudaMalloc fake_malloc
#define cudaMemcpy fake_memcpy
#define cudaStreamSynchronize fake_sync
#define cudaFuncSetAttribute fake_attr
#define cudaGetDevice fake_getdev
#define cudaLibraryLoadData fake_libload
#define cudaLibraryGetKernel fake_libkernel
#include "../paper_1812_02459_gb300/csrc/lbm_adjoint.cu"

lbm_status lbm_internal_step(lbm_handle *) { return LBM_OK; }   // not reached: no sweep runs here
lbm_status lbm_internal_poll_device_error(lbm_handle *) { return LBM_OK; }   // not reached either

namespace {

int failures = 0;
#define EXPECT(c, what)                                                   \
    do {                                                                  \
        if (!(c)) {                                                       \
            if (failures < 20) printf("  FAIL %s (%s:%d)\n", what, __FILE__, __LINE__); \
            ++failures;                                                   \
        }                                                                 \
    } while (0)

lbm_params params(int flux, int picard, int filter)
{
    lbm_params P{};
    P.M = 0.1; P.eta = 2.0; P.W = 4.0; P.sigma = 5e-3; P.lambda = 0.005; P.flux_correction = flux;
    P.rho_H = 100; P.rho_L = 1; P.nu_H = 0.1; P.nu_L = 0.1;
    const double sf[9] = {1, 1, 1, 1, 1, 1, 1, 1, 1}, sg[9] = {1, 1, 1, 1, 1.7, 1, 1.7, 1, 1};
    for (int i = 0; i < 9; ++i) { P.s_f[i] = sf[i]; P.s_g[i] = sg[i]; }
    P.filter_order = filter; P.filter_a = 0.5; P.picard_iters = picard; P.grad_eps = 1e-4;
    return P;
}

template <typename T> void check_case(int flux, int picard, int filter, bool nvrtc, int perx = 1, int pery = 1)
{
    const lbm_params P = params(flux, picard, filter);
    Engine<T> E;
    E.nx = 40; E.ny = 24; E.N = 40 * 24; E.nb = 1;
    E.perx = perx; E.pery = pery;
    E.stencils = make_stencils(P);
    Recorder<T> R(E, P);
    static T src[1], lam[1];
    StateIds in;
    for (int i = 0; i < NSTATE; ++i) *slot(in, i) = E.leaf(src);
    StateIds out = R.step(in);
    for (int i = 0; i < NSTATE; ++i) E.seed(*slot(out, i), lam);
    E.Bwant = 4;
    E.schedule();
    EXPECT(E.err == cudaSuccess, "schedule");
    // forward kernels
    for (auto &G : E.fgroups)
        for (int j = 0; j < G.n; ++j) {
            const VOp<T> &d = E.hfwd[G.off + j];
            for (int i = 0; i < d.nin; ++i) {
                if ((d.fint >> i) & 1u) EXPECT(d.fslot[i] >= 0 && d.fslot[i] < G.slots, "forward input slot");
                else EXPECT(d.in[i] != nullptr, "forward global input has storage");
            }
            if (d.k == OP_STENCIL) EXPECT(d.fint == 0, "stencil input from a complete plane");
            if (d.fout >= 0) EXPECT(d.fout < G.slots, "forward output slot");
        }
    // reverse kernels: records, staging, flushes
    for (auto &G : E.rgroups) {
        for (int p = 0; p < G.nph; ++p) {
            const VPhase &Ph = E.hph[G.ph0 + p];
            EXPECT(Ph.o0 >= 0 && Ph.o0 + Ph.no <= G.nops && Ph.e0 >= 0 && Ph.e0 + Ph.ne <= G.npre, "phase ranges");
            std::map<int, int> staged;
            for (int e = Ph.e0; e < Ph.e0 + Ph.ne; ++e) {
                const VPre<T> &V = E.hpre[G.pre0 + e];
                EXPECT(V.slot >= 0 && V.slot < G.slots, "staging slot");
                EXPECT(V.p != nullptr, "staged plane has storage");
                EXPECT(staged.count(V.slot) == 0, "staging slot used once per phase");
                staged[V.slot] = 1;
            }
            for (int o = Ph.o0; o < Ph.o0 + Ph.no; ++o) {
                const VRop<T> &r = E.hrop[G.op0 + o];
                for (int i = 0; i < r.nc; ++i) {
                    EXPECT(r.rslot[i] >= 0 && r.rslot[i] < G.slots, "contribution slot");
                    EXPECT(staged.count(r.rslot[i]) == 0, "contribution slot is not a staging slot");
                }
                if (r.rout >= 0) EXPECT(r.rout < G.slots, "in-kernel output adjoint slot");
                const short sv[4] = {r.sa, r.sb, r.sz, r.sg};
                for (short v : sv)
                    if (v >= 0) EXPECT(staged.count(v) == 1, "operand staged in its phase");
                if (r.k == OP_STENCIL)
                    for (int j = 0; j < E.stencils[r.st].n; ++j) EXPECT(staged.count(r.stap + j) == 1, "tap staged");
                if (r.k != OP_LIN && r.k != OP_SQRT && r.k != OP_STENCIL) EXPECT(r.sa >= 0, "value a staged");
                if (r.k == OP_MUL || r.k == OP_DIV) EXPECT(r.sb >= 0, "value b staged");
                if (r.k == OP_SQRT) EXPECT(r.sz >= 0, "value z staged");
            }
        }
        for (int j = 0; j < G.nfl; ++j) {
            const VFlush<T> &F = E.hfl[G.fl0 + j];
            EXPECT(F.slot >= 0 && F.slot < G.slots && F.dst != nullptr, "flush");
        }
    }
    for (auto &l : E.leaves) EXPECT(E.val[l.first] != nullptr, "leaf stored");
    // walls: every stencil's ghost signs are parities or zero, the bounce-back
    // masks appear exactly when an axis is walled (two per direction of f and g)
    int masks = 0, zero_ghost = 0;
    for (const Op &o : E.tape) {
        if (o.k != OP_STENCIL) continue;
        EXPECT(o.sgx >= -1 && o.sgx <= 1 && o.sgy >= -1 && o.sgy <= 1, "ghost signs");
        if (E.stencils[o.st].mask) ++masks;
        if (o.sgx == 0 && o.sgy == 0) ++zero_ghost;
    }
    EXPECT(masks == (E.walls() ? 18 : 0), "bounce-back masks");
    EXPECT(zero_ghost == (E.walls() ? 18 : 0), "streaming shifts with zero ghosts");
    int ids[NSTATE], ido[NSTATE];
    for (int i = 0; i < NSTATE; ++i) {
        ids[i] = *slot(in, i);
        ido[i] = *slot(out, i);
        EXPECT(E.flowed[ids[i]], "every input state plane reached by the sweep");
    }
    if (nvrtc) {
        EXPECT(E.jit, "generated level kernels compile");
        EXPECT(E.enable_pingpong(ids, ido, NSTATE), "argument packs can be exchanged");
        for (auto &J : E.jrev) EXPECT(J.pack_sw.size() == J.pack.size(), "exchanged pack");
    }
    printf("%s flux %d picard %d filter %2d walls %d%d: %zu ops, %zu forward + %zu reverse kernels, compiled %d, "
           "failures %d\n",
           sizeof(T) == 8 ? "fp64" : "fp32", flux, picard, filter, !perx, !pery, E.tape.size(), E.fgroups.size(),
           E.rgroups.size(), (int)E.jit, failures);
}

}  // namespace

int main(int argc, char **argv)
{
    const bool nvrtc = argc > 1 && argv[1][0] == '1' && lbm_jit::nvrtc().ok;
    const int cases[][3] = {{1, 2, 11}, {0, 2, 11}, {1, 1, 0}, {1, 3, 5}, {0, 1, 7}};
    for (auto &c : cases) {
        check_case<float>(c[0], c[1], c[2], nvrtc);
        if (failures) return 1;
    }
    check_case<double>(1, 2, 11, nvrtc);
    // walls in y, in x and y (FP32), in y (FP64)
    check_case<float>(1, 2, 11, nvrtc, 1, 0);
    check_case<float>(1, 2, 11, nvrtc, 0, 0);
    check_case<double>(1, 2, 11, nvrtc, 1, 0);
    return failures ? 1 : 0;
}
