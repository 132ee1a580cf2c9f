// lbm_internal.h -- the handle behind the C ABI, shared by the library's
// translation units (not installed, not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_kernels.cuh"

struct lbm_adjoint;   // reverse-mode state, lbm_adjoint.cu

struct lbm_handle {
    lbm_grid grid{};
    lbm_params prm{};
    cudaStream_t stream = nullptr;
    std::string err;
    long long N = 0;
    size_t elem = 0, pop_elem = 0;     // bytes of T and of S
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    void *f[2]{}, *g[2]{};
    int cur = 0;                       // which population buffer holds the state
    void *phi[2]{};                    // phi[pcur] = phi^n; the other slot holds the phi of the
    int pcur = 0;                      // previous step until the RK3 pass writes phi^{n+1} there
    void *philo = nullptr;             // FP32 arithmetic: phi = phi[pcur] + philo (float pair)
    void *pf = nullptr, *ux[2]{}, *uy[2]{};
    int ucur = 0;                      // ux[ucur] = filtered u^n, ux[1-ucur] = u^{n-1}
    void *uhx = nullptr, *uhy = nullptr;
    void *dbar[2]{}, *phat[2]{};       // post-stream moments, double-buffered: dbar = phi_bar - phi
    int acur = 0;                      // of the collision; slot acur = moments of the stored populations
    void *jx = nullptr, *jy = nullptr;
    void *s1 = nullptr, *s2 = nullptr, *tk[2][2]{};
    double *diag_part = nullptr, *diag_out = nullptr;
    int diag_blocks = 1;
    lbm::KP<double> kpd{};
    lbm::KP<float> kpf{};
    // per-kernel timing; inside lbm_step a launch that directly follows
    // another timed launch starts at that one's end event (chain), so a
    // step records one event per launch boundary
    bool prof = false;
    bool chain_ok = false;
    cudaEvent_t chain = nullptr;
    struct Mark { int kind; cudaEvent_t a, b; bool own_a; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> pool;
    double prof_ms[LBM_NKERNELS]{};
    long long prof_n[LBM_NKERNELS]{};
    // true while the state is exactly the initialisation from fields
    // (lbm_create / lbm_set_fields, no step since): the adjoint needs it
    bool fresh_init = false;
    lbm_adjoint *adj = nullptr;
    // TMA tile staging (FP32 arithmetic, nx a multiple of 4): tensor maps
    // by (plane, window) and the device word that bounded waits report to
    struct TmaEntry {
        const void *ptr;
        int bw, bh;
        CUtensorMap map;
    };
    bool tma = false;
    std::vector<TmaEntry> tmaps;
    unsigned *dev_err = nullptr;
    // set once a synchronising call has seen *dev_err != 0; sticky: lbm_step
    // refuses to run on such a handle
    bool failed = false;
    // periodic check of lbm_set_check: every chk_every steps the sums go to
    // page-locked chk_host behind event chk_ev; a later lbm_step reads them
    int chk_every = 0;
    double chk_delta = 0.0;
    long long chk_count = 0;
    double *chk_host = nullptr;
    cudaEvent_t chk_ev = nullptr;
    bool chk_pending = false;
    lbm_status chk_status = LBM_OK;
};

// After a synchronisation of the handle's stream: LBM_ERR_CUDA (and the
// sticky failed flag) if a kernel gave up a bounded tile-copy wait
// (lbm_api.cu).
lbm_status lbm_internal_poll_device_error(lbm_handle *h);

// The plane of phi^n.
inline void *phi_cur(const lbm_handle *h) { return h->phi[h->pcur]; }

// Issue one step on the handle's stream (lbm_api.cu).
lbm_status lbm_internal_step(lbm_handle *h);
// Free the reverse-mode state (lbm_adjoint.cu).
void lbm_internal_adjoint_free(lbm_handle *h);
