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
    void *phi = nullptr, *pf = nullptr, *ux[2]{}, *uy[2]{};
    int ucur = 0;                      // ux[ucur] = filtered u^n, ux[1-ucur] = u^{n-1}
    void *uhx = nullptr, *uhy = nullptr;
    void *phibar[2]{}, *phat[2]{};     // post-stream moments, double-buffered:
    int acur = 0;                      // slot acur = moments of the stored populations
    void *jx = nullptr, *jy = nullptr;
    void *s1 = nullptr, *s2 = nullptr, *tk[2][2]{};
    double *diag_part = nullptr, *diag_out = nullptr;
    int diag_blocks = 1;
    lbm::KP<double> kpd{};
    lbm::KP<float> kpf{};
    // per-kernel timing
    bool prof = false;
    struct Mark { int kind; cudaEvent_t a, b; };
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
};

// Issue one step on the handle's stream (lbm_api.cu).
lbm_status lbm_internal_step(lbm_handle *h);
// Free the reverse-mode state (lbm_adjoint.cu).
void lbm_internal_adjoint_free(lbm_handle *h);
