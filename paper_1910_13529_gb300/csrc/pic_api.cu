// C ABI of libpic (include/pic.h): handle lifecycle, validation, scratch ownership and the
// ordering of the kernels that make up one PIC step (Sec. 1 loop of arXiv:1910.13529).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <algorithm>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct SpeciesSlot {
    bool bound = false;
    int32_t* cell = nullptr;
    float* off = nullptr;
    float* u = nullptr;
    int32_t* id = nullptr;
    long long cap = 0;
    long long extent = 0;      // upper bound of the device count
    double q = 0, m = 1, w = 0;
    int32_t* prev_cell = nullptr;   // library scratch for the unfused path
    float* prev_off = nullptr;
    int32_t* defer = nullptr;       // 3D fused path: list of chunks left to the global-memory kernel
};

struct pic_t {
    pic_config cfg;
    GridP g;
    StencilP st;
    double C64[PIC_MAX_M];        // E-side d+ coefficients
    double C64b[PIC_MAX_M];       // B-side d- coefficients (= C64 unless split)
    bool split = false;
    double h64[2 * PIC_MAX_HLEN + 1];
    float hf[2 * PIC_MAX_HLEN + 1];
    int hlen = 0;
    int device = 0;
    float* E = nullptr;
    float* B = nullptr;
    float* J = nullptr;
    // scratch owned by the library
    float* E2 = nullptr;
    float* B2 = nullptr;
    double* rho64 = nullptr;
    double* acc = nullptr;
    int* status = nullptr;
    int32_t* counts = nullptr;
    int32_t* hist = nullptr;
    int32_t* blocksums = nullptr;
    int32_t* cell_alt = nullptr;
    float* off_alt = nullptr;
    float* u_alt = nullptr;
    int32_t* id_alt = nullptr;
    long long alt_cap = 0;
    SpeciesSlot sp[PIC_MAX_SPECIES];
    long long step = 0, shifts = 0, next_id = 0;
    int pending_shift = 0;
    int state = 0;   // 0: idle, 1: pushed (unfused), 2: deposited
    char err[256] = {0};
    // kernel timing
    bool timing = false;
    std::vector<cudaEvent_t> ev_a, ev_b;
    std::vector<int> ev_cat;
    size_t ev_used = 0;
    long long launches[PIC_TIMING_N] = {0};
    float* adj_scratch = nullptr; // adjoint: B', E', W (7 N floats)
    double* static_rho = nullptr; // device address of g_static_rho on this handle's device
    int fa_variant = 0;           // field-advance tile variant (pic_autotune)
    KSpaceState* ks = nullptr;    // k-space solvers: transforms, buffers and symbol tables
    double fa_ms[PIC_MAX_TILE_VARIANTS] = {0};   // measured time per variant (ms), 0 = not measured
};

namespace {

char g_create_err[256] = "no error";

// Fixed FP64 charge-density scratch of pic_gauss_static (no allocation).  In host code the
// name g_static_rho is only a stand-in: pic_create looks up its device address with
// cudaGetSymbolAddress, with the handle's device current, and keeps it in the handle.  Under
// lazy module loading that lookup is what loads this module (and places the array) on the
// device, so it happens when the handle is created, where allocation is expected, and never in
// pic_gauss_static itself.
__device__ __align__(256) double g_static_rho[PIC_STATIC_RHO_CELLS];

pic_status fail(pic_t* h, pic_status st, const char* fmt, ...) {
    char* dst = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 256, fmt, ap);
    va_end(ap);
    return st;
}

pic_status cuda_fail(pic_t* h, cudaError_t e, const char* what) {
    return fail(h, PIC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, call, what)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, what); \
    } while (0)

template <typename T>
pic_status dalloc(pic_t* h, T** p, size_t n, const char* what) {
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * (n ? n : 1));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(h, PIC_ERR_OOM, "cudaMalloc %s (%zu bytes): %s", what, sizeof(T) * n, cudaGetErrorString(e));
    }
    return PIC_OK;
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

// Brackets one kernel class on the stream with a pair of events while timing is on.
struct Scope {
    pic_t* h;
    cudaStream_t s;
    size_t i;
    bool on;
    Scope(pic_t* h_, int cat, int nlaunch, cudaStream_t s_) : h(h_), s(s_), i(0), on(h_->timing) {
        h->launches[cat] += nlaunch;
        if (!on) return;
        if (h->ev_used == h->ev_a.size()) {
            cudaEvent_t a, b;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
                on = false;
                return;
            }
            h->ev_a.push_back(a);
            h->ev_b.push_back(b);
            h->ev_cat.push_back(cat);
        }
        i = h->ev_used++;
        h->ev_cat[i] = cat;
        cudaEventRecord(h->ev_a[i], s);
    }
    ~Scope() {
        if (on) cudaEventRecord(h->ev_b[i], s);
    }
};

SpeciesP species_params(pic_t* h, int s) {
    SpeciesSlot& q = h->sp[s];
    SpeciesP p;
    p.cell = q.cell;
    p.off = q.off;
    p.u = q.u;
    p.id = q.id;
    p.count = h->counts + s;
    p.cap = q.cap;
    double V = h->cfg.dz * h->cfg.dx * (h->cfg.ndim == 3 ? h->cfg.dy : 1.0);
    p.eps = (float)(q.q * h->cfg.dt / (2.0 * q.m));
    const double k3[3] = {h->cfg.dt / h->cfg.dz, h->cfg.dt / h->cfg.dx, h->cfg.dt / h->cfg.dy};
    float* dst[3] = {p.kz, p.kx, p.ky};
    for (int a = 0; a < 3; ++a) {
        dst[a][0] = (float)k3[a];
        dst[a][1] = (float)(k3[a] - (double)dst[a][0]);
    }
    p.qv64 = q.q * q.w / V;
    p.qv = (float)p.qv64;
    p.wm = q.w * q.m;
    p.prev_cell = q.prev_cell;
    p.prev_off = q.prev_off;
    return p;
}

bool window_due(const pic_t* h, long long steps_done) {
    if (!h->cfg.moving_window) return false;
    return (long long)std::floor(steps_done * h->cfg.dt / h->cfg.dz + 1e-9) > h->shifts;
}

pic_status need_fields(pic_t* h) {
    if (!h->E || !h->B || !h->J) return fail(h, PIC_ERR_STATE, "fields not bound (pic_bind_fields)");
    return PIC_OK;
}

// Field advance from (Ein, Bin) into (Eout, Bout), with the window shift and injection that
// complete step n.  J1 has already been corrected in place for the customised stencil.
pic_status advance_fields(pic_t* h, const float* Ein, const float* Bin, float* Eout, float* Bout,
                          cudaStream_t s) {
    const long long N = h->g.ncell;
    const long long n_done = h->step + 1;
    const int shift = window_due(h, n_done) ? 1 : 0;
    FieldP p;
    p.g = h->g;
    p.st = h->st;
    p.Ein = Ein;
    p.Bin = Bin;
    p.J1 = h->J;
    p.J2 = h->J + N;
    p.J3 = h->J + 2 * N;
    p.Eout = Eout;
    p.Bout = Bout;
    p.shift = shift;
    if (h->ks) {
        Scope sc(h, PIC_T_FIELDS, 1, s);
        char kerr[256] = {0};
        if (kspace_advance(h->ks, Ein, Bin, h->J, Eout, Bout, s, kerr, sizeof kerr))
            return fail(h, PIC_ERR_CUDA, "%s", kerr);
    } else {
        Scope sc(h, PIC_T_FIELDS, 1, s);
        CK(h, launch_field_advance(p, s, h->fa_variant), "field advance kernel");
    }
    h->step = n_done;
    if (shift) {
        h->shifts += 1;
        h->pending_shift = 1;
        int is = h->cfg.inject_species;
        if (is >= 0 && h->sp[is].bound) {
            SpeciesP sp = species_params(h, is);
            {
                Scope sc(h, PIC_T_WINDOW, 2, s);
                CK(h, launch_inject(h->g, sp, h->cfg.inject_ppc, h->next_id, h->status, &h->sp[is].extent, s),
                   "inject kernel");
            }
            long long nnew = (long long)h->cfg.nx * (h->cfg.ndim == 3 ? h->cfg.ny : 1) * h->cfg.inject_ppc[0] *
                             h->cfg.inject_ppc[1] * (h->cfg.ndim == 3 ? h->cfg.inject_ppc[2] : 1);
            h->next_id += nnew;
        }
    }
    return PIC_OK;
}

// After the deposit: the current filter on J1, J2, J3 and the Sec. 3 correction on J1, fused
// into one launch when both are configured.
pic_status smooth_current(pic_t* h, cudaStream_t s) {
    if (h->cfg.current_filter && h->hlen > 0) {
        Scope sc(h, PIC_T_FILTER, 1, s);
        CK(h, launch_filter_correct(h->g, h->hf, h->hlen, h->J, s), "current filter + correction kernel");
    } else if (h->cfg.current_filter) {
        Scope sc(h, PIC_T_FILTER, 1, s);
        CK(h, launch_filter_current(h->g, h->J, s), "current filter kernel");
    } else if (h->hlen > 0) {
        Scope sc(h, PIC_T_CORRECTION, 1, s);
        CK(h, launch_correct_j1(h->g, h->hf, h->hlen, h->J, s), "current correction kernel");
    }
    return PIC_OK;
}

pic_status ensure_sort_scratch(pic_t* h) {
    long long cap = 0;
    bool ids = false;
    for (auto& q : h->sp)
        if (q.bound) {
            cap = q.cap > cap ? q.cap : cap;
            ids = ids || q.id;
        }
    if (!h->hist) {
        long long nb = sort_bins(h->g);
        pic_status st = dalloc(h, &h->hist, nb, "sort histogram");
        if (st) return st;
        if ((st = dalloc(h, &h->blocksums, nb / 4096 + 16, "sort block sums"))) return st;
    }
    if (cap > h->alt_cap) {
        dfree(h->cell_alt);
        dfree(h->off_alt);
        dfree(h->u_alt);
        dfree(h->id_alt);
        h->cell_alt = nullptr;
        h->off_alt = h->u_alt = nullptr;
        h->id_alt = nullptr;
        h->alt_cap = 0;
        pic_status st;
        if ((st = dalloc(h, &h->cell_alt, cap, "sort cells"))) return st;
        if ((st = dalloc(h, &h->off_alt, cap * h->cfg.ndim, "sort offsets"))) return st;
        if ((st = dalloc(h, &h->u_alt, cap * 3, "sort momenta"))) return st;
        if ((st = dalloc(h, &h->id_alt, cap, "sort ids"))) return st;
        h->alt_cap = cap;
    }
    return PIC_OK;
}

pic_status do_sort(pic_t* h, cudaStream_t s) {
    pic_status st = ensure_sort_scratch(h);
    if (st) return st;
    for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
        if (!h->sp[i].bound) continue;
        SpeciesP sp = species_params(h, i);
        // the alternate arrays use the species' own capacity as component stride
        Scope sc(h, PIC_T_SORT, 8, s);
        CK(h, launch_sort(h->g, sp, h->sp[i].extent, h->hist, h->blocksums, h->cell_alt, h->off_alt,
                          h->u_alt, h->id_alt, s),
           "sort kernels");
    }
    return PIC_OK;
}

}  // namespace

extern "C" {

const char* pic_last_error(const pic_t* h) { return h ? h->err : g_create_err; }

pic_status pic_fit_coefficients(double kappa, int M, double wk, double n, double* C_out) {
    if (!C_out || M < 1 || M > PIC_MAX_M || !(kappa > 0.0)) return PIC_ERR_ARG;
    return fit_coefficients(kappa, M, wk, n, C_out) ? PIC_ERR_ARG : PIC_OK;
}

pic_status pic_fit_coefficients_b(double kappa, int M, double wk, double n, const double* CE, int ME,
                                  double* C_out) {
    if (!C_out || !CE || M < 1 || M > PIC_MAX_M || ME < 1 || ME > PIC_MAX_M || !(kappa > 0.0)) return PIC_ERR_ARG;
    return fit_coefficients_b(kappa, M, wk, n, CE, ME, C_out) ? PIC_ERR_ARG : PIC_OK;
}

pic_status pic_correction_taps(const double* C, int M, int hlen, double* h_out) {
    if (!C || !h_out || M < 1 || M > PIC_MAX_M || hlen < 0 || hlen > 4096) return PIC_ERR_ARG;
    return correction_taps(C, M, hlen, h_out) ? PIC_ERR_ARG : PIC_OK;
}

pic_status pic_cfl_dt_split(int ndim, double dz, double dx, double dy, const double* CE, const double* CB, int M,
                            double* dt_out) {
    if (!dt_out || !CE || !CB || M < 1 || M > PIC_MAX_M || (ndim != 2 && ndim != 3) || !(dz > 0) || !(dx > 0) ||
        (ndim == 3 && !(dy > 0)))
        return PIC_ERR_ARG;
    const double dt = cfl_dt_split(ndim, dz, dx, dy, CE, CB, M);
    if (dt < 0.0) return PIC_ERR_ARG;
    *dt_out = dt;
    return PIC_OK;
}

pic_status pic_cfl_dt_kspace(int ndim, int solver, double dz, double dx, double dy, double* dt_out) {
    if (!dt_out || (solver != PIC_SOLVER_SPECTRAL && solver != PIC_SOLVER_KT && solver != PIC_SOLVER_PSATD) ||
        (ndim != 2 && ndim != 3) || !(dz > 0) || !(dx > 0) || (ndim == 3 && !(dy > 0)))
        return PIC_ERR_ARG;
    *dt_out = kspace_cfl_dt(ndim, solver == PIC_SOLVER_PSATD ? 2 : solver == PIC_SOLVER_KT ? 1 : 0, dz, dx, dy);
    return PIC_OK;
}

pic_status pic_cfl_dt(int ndim, double dz, double dx, double dy, const double* C, int M, double* dt_out) {
    if (!dt_out || !C || M < 1 || M > PIC_MAX_M || (ndim != 2 && ndim != 3) || !(dz > 0) || !(dx > 0) ||
        (ndim == 3 && !(dy > 0)))
        return PIC_ERR_ARG;
    *dt_out = cfl_dt(ndim, dz, dx, dy, C, M);
    return PIC_OK;
}

pic_status pic_create(const pic_config* cfg, pic_t** out) {
    if (!cfg || !out) return fail(nullptr, PIC_ERR_ARG, "null argument");
    *out = nullptr;
    const pic_config& c = *cfg;
    if (c.ndim != 2 && c.ndim != 3) return fail(nullptr, PIC_ERR_ARG, "ndim must be 2 or 3");
    int ny = c.ndim == 3 ? c.ny : 1;
    if (c.nz < 4 || c.nx < 4 || (c.ndim == 3 && c.ny < 4))
        return fail(nullptr, PIC_ERR_ARG, "grid too small (nz, nx, ny >= 4)");
    if ((long long)(c.nz + 2) * c.nx * ny >= (1LL << 31) - 1)
        return fail(nullptr, PIC_ERR_ARG, "grid too large for 32-bit cell indices");
    if (c.nz > 32768) return fail(nullptr, PIC_ERR_ARG, "nz above 32768");
    if (!(c.dz > 0) || !(c.dx > 0) || (c.ndim == 3 && !(c.dy > 0)) || !(c.dt > 0))
        return fail(nullptr, PIC_ERR_ARG, "cell sizes and dt must be positive");
    if (c.solver != PIC_SOLVER_YEE && c.solver != PIC_SOLVER_CUSTOM && c.solver != PIC_SOLVER_SPECTRAL &&
        c.solver != PIC_SOLVER_KT && c.solver != PIC_SOLVER_PSATD)
        return fail(nullptr, PIC_ERR_ARG, "unknown solver %d", c.solver);
    const bool kspace = c.solver == PIC_SOLVER_SPECTRAL || c.solver == PIC_SOLVER_KT || c.solver == PIC_SOLVER_PSATD;
    const int kkind = c.solver == PIC_SOLVER_PSATD ? 2 : c.solver == PIC_SOLVER_KT ? 1 : 0;
    if (kspace) {
        if (!kspace_available())
            return fail(nullptr, PIC_ERR_ARG, "k-space solvers need cuFFT, which this build does not have");
        if (c.moving_window) return fail(nullptr, PIC_ERR_ARG, "k-space solvers are periodic along z: no moving window");
        if (c.coef_b) return fail(nullptr, PIC_ERR_ARG, "coef_b is for the customised solver");
    }
    if (c.shape != 1 && c.shape != 2) return fail(nullptr, PIC_ERR_ARG, "shape must be 1 or 2");
    if (c.precision != 0 && c.precision != 32)
        return fail(nullptr, PIC_ERR_ARG, "precision %d: only FP32 (0 or 32) kernels are built", c.precision);
    if (c.current_filter != PIC_FILTER_NONE && c.current_filter != PIC_FILTER_5PASS)
        return fail(nullptr, PIC_ERR_ARG, "unknown current_filter %d", c.current_filter);
    if (c.inject_species >= PIC_MAX_SPECIES) return fail(nullptr, PIC_ERR_ARG, "inject_species out of range");
    if (c.inject_species >= 0 && (c.inject_ppc[0] < 1 || c.inject_ppc[1] < 1 || (c.ndim == 3 && c.inject_ppc[2] < 1)))
        return fail(nullptr, PIC_ERR_ARG, "inject_ppc must be >= 1");
    int M = 1;
    double C[PIC_MAX_M] = {1.0};
    double CB[PIC_MAX_M] = {1.0};
    if (c.coef_b && (c.solver != PIC_SOLVER_CUSTOM || !c.coef))
        return fail(nullptr, PIC_ERR_ARG, "coef_b needs the customised solver with explicit coef");
    if (c.solver == PIC_SOLVER_CUSTOM) {
        M = c.M;
        if (M < 1 || M > PIC_MAX_M) return fail(nullptr, PIC_ERR_ARG, "M must be in [1, %d]", PIC_MAX_M);
        if (c.coef) {
            for (int l = 0; l < M; ++l) C[l] = c.coef[l];
        } else if (fit_coefficients(c.dz / c.dt, M, c.fit_wk, c.fit_n, C)) {
            return fail(nullptr, PIC_ERR_ARG, "coefficient fit failed");
        }
        for (int l = 0; l < M; ++l) CB[l] = c.coef_b ? c.coef_b[l] : C[l];
    }
    const bool split = c.coef_b != nullptr;
    double dtmax = kspace ? kspace_cfl_dt(c.ndim, kkind, c.dz, c.dx, c.ndim == 3 ? c.dy : 1.0)
                          : cfl_dt_split(c.ndim, c.dz, c.dx, c.dy, C, CB, M);
    if (dtmax < 0.0) return fail(nullptr, PIC_ERR_ARG, "[k]_E1 [k]_B1 changes sign: unstable for every dt");
    if (c.dt > dtmax * (1.0 + 1e-12))
        return fail(nullptr, PIC_ERR_CFL, "dt = %.6g above the stability limit %.6g", c.dt, dtmax);

    pic_t* h = new (std::nothrow) pic_t();
    if (!h) return fail(nullptr, PIC_ERR_OOM, "host allocation");
    h->cfg = c;
    h->cfg.ny = ny;
    h->cfg.coef = nullptr;
    h->cfg.coef_b = nullptr;
    h->split = split;
    if (c.ndim == 2) h->cfg.dy = 1.0;
    cudaGetDevice(&h->device);
    GridP& g = h->g;
    g.ndim = c.ndim;
    g.nz = c.nz;
    g.nx = c.nx;
    g.ny = ny;
    g.nzg = c.nz + 2;
    g.ncell = (long long)c.nz * c.nx * ny;
    g.dz = (float)c.dz;
    g.dx = (float)c.dx;
    g.dy = (float)h->cfg.dy;
    g.dt = (float)c.dt;
    g.shape = c.shape;
    h->st.M = M;
    h->fa_variant = default_field_variant(c.ndim, M);
    bool yee_b = true;     // B-side d- is the two-point Yee difference: no correction
    for (int l = 0; l < PIC_MAX_M; ++l) {
        h->C64[l] = l < M ? C[l] : 0.0;
        h->C64b[l] = l < M ? CB[l] : 0.0;
        h->st.C[l] = (float)h->C64[l];
        h->st.Cm[l] = (float)h->C64b[l];
        yee_b = yee_b && h->C64b[l] == (l == 0 ? 1.0 : 0.0);
    }
    // Sec. 3 correction: P = [k]_B1 / [k]_Yee, from the B-side coefficients
    if (c.solver == PIC_SOLVER_CUSTOM && (split ? !yee_b : M > 1)) {
        h->hlen = PIC_MAX_HLEN;
        if (correction_taps(CB, M, h->hlen, h->h64)) {
            delete h;
            return fail(nullptr, PIC_ERR_ARG, "stencil symbol ratio has a zero: no current correction");
        }
        for (int i = 0; i < 2 * h->hlen + 1; ++i) h->hf[i] = (float)h->h64[i];
    }
    const long long N = g.ncell;
    pic_status st;
    if ((st = dalloc(h, &h->E2, 3 * N, "field buffer E")) || (st = dalloc(h, &h->B2, 3 * N, "field buffer B")) ||
        (st = dalloc(h, &h->rho64, N, "rho")) || (st = dalloc(h, &h->acc, 16, "diag accumulators")) ||
        (st = dalloc(h, &h->status, 1, "status")) || (st = dalloc(h, &h->counts, PIC_MAX_SPECIES, "counts"))) {
        snprintf(g_create_err, sizeof g_create_err, "%s", h->err);
        pic_destroy(h);
        return st;
    }
    if (kspace) {
        char kerr[256] = {0};
        const int r = kspace_create(g, c.solver, c.dz, c.dx, h->cfg.dy, c.dt, &h->ks, kerr, sizeof kerr);
        if (r) {
            snprintf(g_create_err, sizeof g_create_err, "%s", kerr);
            pic_destroy(h);
            return r == 2 ? PIC_ERR_OOM : PIC_ERR_CUDA;
        }
    }
    cudaError_t e = cudaMemset(h->status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(h->counts, 0, sizeof(int32_t) * PIC_MAX_SPECIES);
    if (e == cudaSuccess) {
        void* ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_rho);
        h->static_rho = static_cast<double*>(ptr);
    }
    if (e != cudaSuccess) {
        snprintf(g_create_err, sizeof g_create_err, "cudaMemset: %s", cudaGetErrorString(e));
        pic_destroy(h);
        return PIC_ERR_CUDA;
    }
    *out = h;
    return PIC_OK;
}

pic_status pic_destroy(pic_t* h) {
    if (!h) return PIC_OK;
    void* ptrs[] = {h->E2, h->B2, h->rho64, h->acc, h->status, h->counts, h->hist, h->blocksums,
                    h->cell_alt, h->off_alt, h->u_alt, h->id_alt};
    for (void* p : ptrs) dfree(p);
    dfree(h->adj_scratch);
    kspace_destroy(h->ks);
    for (size_t i = 0; i < h->ev_a.size(); ++i) {
        cudaEventDestroy(h->ev_a[i]);
        cudaEventDestroy(h->ev_b[i]);
    }
    for (auto& q : h->sp) {
        dfree(q.prev_cell);
        dfree(q.prev_off);
        dfree(q.defer);
    }
    delete h;
    return PIC_OK;
}

pic_status pic_get_coefficients_b(const pic_t* h, double* Cb_out, int* split) {
    if (!h) return PIC_ERR_ARG;
    if (Cb_out)
        for (int l = 0; l < PIC_MAX_M; ++l) Cb_out[l] = h->C64b[l];
    if (split) *split = h->split ? 1 : 0;
    return PIC_OK;
}

pic_status pic_get_coefficients(const pic_t* h, double* C_out, int* M, double* h_out, int* hlen) {
    if (!h) return PIC_ERR_ARG;
    if (C_out)
        for (int l = 0; l < PIC_MAX_M; ++l) C_out[l] = h->C64[l];
    if (M) *M = h->st.M;
    if (h_out)
        for (int i = 0; i < 2 * PIC_MAX_HLEN + 1; ++i) h_out[i] = i < 2 * h->hlen + 1 ? h->h64[i] : 0.0;
    if (hlen) *hlen = h->hlen;
    return PIC_OK;
}

pic_status pic_bind_fields(pic_t* h, float* E, float* B, float* J) {
    if (!h) return PIC_ERR_ARG;
    if (!E || !B || !J) return fail(h, PIC_ERR_ARG, "null field pointer");
    h->E = E;
    h->B = B;
    h->J = J;
    return PIC_OK;
}

pic_status pic_bind_species(pic_t* h, int s, int32_t* cell, float* off, float* u, int32_t* id, int64_t n,
                            int64_t cap, double q, double m, double w) {
    if (!h) return PIC_ERR_ARG;
    if (s < 0 || s >= PIC_MAX_SPECIES) return fail(h, PIC_ERR_ARG, "species index %d out of range", s);
    if (!cell || !off || !u) return fail(h, PIC_ERR_ARG, "null particle pointer");
    if (n < 0 || cap < n || cap > (1LL << 31) - 1) return fail(h, PIC_ERR_ARG, "need 0 <= n <= cap < 2^31");
    if (!(m > 0)) return fail(h, PIC_ERR_ARG, "mass must be positive");
    SpeciesSlot& sl = h->sp[s];
    dfree(sl.prev_cell);
    dfree(sl.prev_off);
    dfree(sl.defer);
    sl = SpeciesSlot();
    sl.bound = true;
    sl.cell = cell;
    sl.off = off;
    sl.u = u;
    sl.id = id;
    sl.cap = cap;
    sl.extent = n;
    sl.q = q;
    sl.m = m;
    sl.w = w;
    int32_t n32 = (int32_t)n;
    CK(h, cudaMemcpy(h->counts + s, &n32, sizeof(int32_t), cudaMemcpyHostToDevice), "count upload");
    if (id && h->next_id < n) h->next_id = n;
    return PIC_OK;
}

pic_status pic_gather_push(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
        SpeciesSlot& q = h->sp[i];
        if (!q.bound) continue;
        if (!q.prev_cell) {
            if ((st = dalloc(h, &q.prev_cell, q.cap, "previous cells"))) return st;
            if ((st = dalloc(h, &q.prev_off, q.cap * h->cfg.ndim, "previous offsets"))) return st;
        }
        SpeciesP sp = species_params(h, i);
        Scope sc(h, PIC_T_PARTICLES, 1, s);
        CK(h, launch_push(h->g, sp, h->E, h->B, nullptr, h->pending_shift, 1, q.extent, nullptr, s), "push kernel");
    }
    h->pending_shift = 0;
    h->state = 1;
    return PIC_OK;
}

pic_status pic_deposit(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    if (h->state != 1) return fail(h, PIC_ERR_STATE, "pic_deposit needs a preceding pic_gather_push");
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = h->g.ncell;
    {
        Scope sc(h, PIC_T_DEPOSIT, 1, s);
        CK(h, cudaMemsetAsync(h->J, 0, sizeof(float) * 3 * N, s), "zero J");
    }
    for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
        if (!h->sp[i].bound) continue;
        SpeciesP sp = species_params(h, i);
        Scope sc(h, PIC_T_DEPOSIT, 1, s);
        CK(h, launch_deposit_unfused(h->g, sp, h->J, h->sp[i].extent, s), "deposit kernel");
    }
    if ((st = smooth_current(h, s))) return st;
    h->state = 2;
    return PIC_OK;
}

pic_status pic_field_advance(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = h->g.ncell;
    if ((st = advance_fields(h, h->E, h->B, h->E2, h->B2, s))) return st;
    Scope sc(h, PIC_T_FIELDS, 2, s);
    CK(h, cudaMemcpyAsync(h->E, h->E2, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy E");
    CK(h, cudaMemcpyAsync(h->B, h->B2, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy B");
    h->state = 0;
    return PIC_OK;
}

pic_status pic_step(pic_t* h, int nsteps, void* stream) {
    if (!h) return PIC_ERR_ARG;
    if (nsteps < 0) return fail(h, PIC_ERR_ARG, "nsteps < 0");
    pic_status st = need_fields(h);
    if (st) return st;
    if (h->state == 1) return fail(h, PIC_ERR_STATE, "pic_step after pic_gather_push without pic_deposit");
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = h->g.ncell;
    float *Ec = h->E, *Bc = h->B, *En = h->E2, *Bn = h->B2;
    for (int it = 0; it < nsteps; ++it) {
        if (h->cfg.sort_every > 0 && h->step % h->cfg.sort_every == 0)
            if ((st = do_sort(h, s))) return st;
        {
            Scope sc(h, PIC_T_DEPOSIT, 1, s);
            CK(h, cudaMemsetAsync(h->J, 0, sizeof(float) * 3 * N, s), "zero J");
        }
        for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
            if (!h->sp[i].bound) continue;
            SpeciesSlot& q = h->sp[i];
            if (h->cfg.ndim == 3 && !q.defer) {
                const long long len = 2 + (q.cap + 255) / 256;       // two lists of this length
                if ((st = dalloc(h, &q.defer, 2 * len, "deferred chunk lists"))) return st;
                CK(h, cudaMemsetAsync(q.defer, 0, sizeof(int32_t) * 2, s), "clear deferred chunk list");
                CK(h, cudaMemsetAsync(q.defer + len, 0, sizeof(int32_t) * 2, s), "clear deferred chunk list");
            }
            SpeciesP sp = species_params(h, i);
            Scope sc(h, PIC_T_PARTICLES, h->cfg.ndim == 3 ? 3 : 1, s);
            CK(h, launch_push(h->g, sp, Ec, Bc, h->J, h->pending_shift, 0, q.extent, q.defer, s),
               "fused push/deposit kernel");
        }
        h->pending_shift = 0;
        if ((st = smooth_current(h, s))) return st;
        if ((st = advance_fields(h, Ec, Bc, En, Bn, s))) return st;
        float* t = Ec;
        Ec = En;
        En = t;
        t = Bc;
        Bc = Bn;
        Bn = t;
    }
    if (Ec != h->E) {
        Scope sc(h, PIC_T_FIELDS, 2, s);
        CK(h, cudaMemcpyAsync(h->E, Ec, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy E");
        CK(h, cudaMemcpyAsync(h->B, Bc, sizeof(float) * 3 * N, cudaMemcpyDeviceToDevice, s), "copy B");
    }
    h->state = 0;
    return PIC_OK;
}

pic_status pic_filter_current(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Scope sc(h, PIC_T_FILTER, 1, s);
    CK(h, launch_filter_current(h->g, h->J, s), "current filter kernel");
    return PIC_OK;
}

pic_status pic_sort(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    if (h->state == 1) return fail(h, PIC_ERR_STATE, "pic_sort between pic_gather_push and pic_deposit");
    return do_sort(h, (cudaStream_t)stream);
}

pic_status pic_rho(pic_t* h, double* rho, void* stream) {
    if (!h || !rho) return PIC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(h, cudaMemsetAsync(rho, 0, sizeof(double) * h->g.ncell, s), "zero rho");
    for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
        if (!h->sp[i].bound) continue;
        SpeciesP sp = species_params(h, i);
        CK(h, launch_rho(h->g, sp, h->pending_shift, rho, h->sp[i].extent, s), "rho kernel");
    }
    return PIC_OK;
}

pic_status pic_gauss(pic_t* h, double* G, void* stream) {
    if (!h || !G) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    if ((st = pic_rho(h, h->rho64, stream))) return st;
    if (h->cfg.current_filter)
        CK(h, launch_filter_rho(h->g, h->rho64, (cudaStream_t)stream), "rho filter kernel");
    CK(h, launch_gauss(h->g, h->st, h->E, h->rho64, h->cfg.rho_bg, G, (cudaStream_t)stream), "gauss kernel");
    return PIC_OK;
}

pic_status pic_gauss_static(pic_t* h, double* G, void* stream) {
    if (!h || !G) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    if (h->g.ncell > PIC_STATIC_RHO_CELLS)
        return fail(h, PIC_ERR_ARG, "pic_gauss_static: grid of %lld nodes exceeds the fixed scratch of %d nodes",
                    h->g.ncell, PIC_STATIC_RHO_CELLS);
    int dev = -1;
    CK(h, cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != h->device)
        return fail(h, PIC_ERR_ARG, "pic_gauss_static: device %d is current, the handle lives on device %d", dev,
                    h->device);
    double* rho = h->static_rho;     // looked up by pic_create on this device
    if (!rho) return fail(h, PIC_ERR_STATE, "pic_gauss_static: fixed scratch address not set");
    cudaStream_t s = (cudaStream_t)stream;
    CK(h, cudaMemsetAsync(rho, 0, sizeof(double) * h->g.ncell, s), "clear the fixed scratch");
    for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
        if (!h->sp[i].bound) continue;
        SpeciesP sp = species_params(h, i);
        CK(h, launch_rho(h->g, sp, h->pending_shift, rho, h->sp[i].extent, s), "rho kernel");
    }
    if (h->cfg.current_filter) CK(h, launch_filter_rho(h->g, rho, s), "rho filter kernel");
    CK(h, launch_gauss(h->g, h->st, h->E, rho, h->cfg.rho_bg, G, s), "gauss kernel");
    return PIC_OK;
}

pic_status pic_diag(pic_t* h, double* out, void* stream) {
    if (!h || !out) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    Scope sc(h, PIC_T_DIAG, 3, s);
    if ((st = pic_rho(h, h->rho64, stream))) return st;
    if (h->cfg.current_filter) CK(h, launch_filter_rho(h->g, h->rho64, s), "rho filter kernel");
    CK(h, cudaMemsetAsync(h->acc, 0, sizeof(double) * 16, s), "zero accumulators");
    int margin = (h->hlen > 0 ? h->st.M + h->hlen + 2 : 2) + (h->cfg.current_filter ? 5 : 0);
    CK(h, launch_diag_reduce(h->g, h->st, h->E, h->B, h->rho64, h->cfg.rho_bg, margin, h->acc, s), "diag kernel");
    for (int i = 0; i < PIC_MAX_SPECIES; ++i) {
        if (!h->sp[i].bound) continue;
        SpeciesP sp = species_params(h, i);
        CK(h, launch_kinetic(h->g, sp, h->sp[i].extent, h->acc, s), "kinetic kernel");
    }
    double acc[16];
    int status = 0;
    CK(h, cudaMemcpyAsync(acc, h->acc, sizeof acc, cudaMemcpyDeviceToHost, s), "read accumulators");
    CK(h, cudaMemcpyAsync(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost, s), "read status");
    CK(h, cudaStreamSynchronize(s), "diag synchronise");
    double V = h->cfg.dz * h->cfg.dx * h->cfg.dy;
    out[PIC_DIAG_GAUSS_MAX] = acc[0];
    out[PIC_DIAG_GAUSS_RMS] = acc[5] > 0 ? std::sqrt(acc[1] / acc[5]) : 0.0;
    out[PIC_DIAG_RHO_MAX] = acc[2];
    out[PIC_DIAG_FIELD_ENERGY] = 0.5 * acc[3] * V;
    out[PIC_DIAG_KINETIC] = acc[4];
    out[PIC_DIAG_COUNT] = acc[6];
    out[PIC_DIAG_STEP] = (double)h->step;
    out[PIC_DIAG_SHIFTS] = (double)h->shifts;
    out[PIC_DIAG_STATUS] = (double)status;
    out[PIC_DIAG_INTERIOR] = acc[5];
    if (status & STATUS_CAPACITY) return fail(h, PIC_ERR_CAPACITY, "particle capacity exceeded during injection");
    return PIC_OK;
}

pic_status pic_get_count(pic_t* h, int s, int64_t* n, void* stream) {
    if (!h || !n || s < 0 || s >= PIC_MAX_SPECIES) return PIC_ERR_ARG;
    int32_t c = 0;
    CK(h, cudaMemcpyAsync(&c, h->counts + s, sizeof c, cudaMemcpyDeviceToHost, (cudaStream_t)stream), "read count");
    CK(h, cudaStreamSynchronize((cudaStream_t)stream), "count synchronise");
    *n = c;
    return PIC_OK;
}

pic_status pic_get_state(const pic_t* h, int64_t* step, int64_t* shifts, int* pending_shift) {
    if (!h) return PIC_ERR_ARG;
    if (step) *step = h->step;
    if (shifts) *shifts = h->shifts;
    if (pending_shift) *pending_shift = h->pending_shift;
    return PIC_OK;
}

pic_status pic_set_state(pic_t* h, int64_t step, int64_t shifts, int pending_shift, int64_t next_id) {
    if (!h || step < 0 || shifts < 0 || next_id < 0 || (pending_shift != 0 && pending_shift != 1)) return PIC_ERR_ARG;
    if (h->state == 1) return fail(h, PIC_ERR_STATE, "pic_set_state between pic_gather_push and pic_deposit");
    h->step = step;
    h->shifts = shifts;
    h->pending_shift = pending_shift;
    h->next_id = next_id;
    return PIC_OK;
}

pic_status pic_get_next_id(const pic_t* h, int64_t* next_id) {
    if (!h || !next_id) return PIC_ERR_ARG;
    *next_id = h->next_id;
    return PIC_OK;
}

pic_status pic_sync(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    CK(h, cudaStreamSynchronize((cudaStream_t)stream), "synchronise");
    int status = 0;
    CK(h, cudaMemcpy(&status, h->status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (status & STATUS_CAPACITY) return fail(h, PIC_ERR_CAPACITY, "particle capacity exceeded during injection");
    return PIC_OK;
}

pic_status pic_timing(pic_t* h, int enable) {
    if (!h) return PIC_ERR_ARG;
    if (enable) {
        h->ev_used = 0;
        for (auto& c : h->launches) c = 0;
    }
    h->timing = enable != 0;
    return PIC_OK;
}

pic_status pic_timing_read(pic_t* h, double* ms, int64_t* launches, void* stream) {
    if (!h) return PIC_ERR_ARG;
    CK(h, cudaStreamSynchronize((cudaStream_t)stream), "timing synchronise");
    double acc[PIC_TIMING_N] = {0};
    for (size_t i = 0; i < h->ev_used; ++i) {
        float t = 0.f;
        CK(h, cudaEventElapsedTime(&t, h->ev_a[i], h->ev_b[i]), "event time");
        acc[h->ev_cat[i]] += t;
    }
    for (int c = 0; c < PIC_TIMING_N; ++c) {
        if (ms) ms[c] = acc[c];
        if (launches) launches[c] = h->launches[c];
    }
    return PIC_OK;
}

pic_status pic_adjoint_step(pic_t* h, const float* E, const float* B, const float* J, float* aE, float* aB,
                            double* grad, void* stream) {
    if (!h || !E || !B || !J || !aE || !aB || !grad) return PIC_ERR_ARG;
    if (h->split) return fail(h, PIC_ERR_ARG, "pic_adjoint_step needs one coefficient set (no coef_b)");
    if (h->ks) return fail(h, PIC_ERR_ARG, "pic_adjoint_step: finite-difference solvers only");
    const long long N = h->g.ncell;
    if (!h->adj_scratch) {
        pic_status st = dalloc(h, &h->adj_scratch, 7 * N, "adjoint scratch");
        if (st) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    float* Bh = h->adj_scratch;        // B' = B - h T E
    float* Ep = Bh + 3 * N;            // E' = E + dt (S B' - J)
    float* W = Ep + 3 * N;             // P^{-1} aE1
    const float dt = h->g.dt, hh = 0.5f * dt;
    const int M = h->st.M;
    const GridP& g = h->g;
    CK(h, launch_curl_plus_update(g, h->st, B, E, -hh, Bh, s), "adjoint: B half step");
    CK(h, launch_curl_minus_update(g, h->st, E, Bh, J, dt, -dt, Ep, s), "adjoint: E step");
    CK(h, launch_grad_plus(g, M, aB, Ep, -(double)hh, grad, s), "adjoint: gradient (third stage)");
    CK(h, launch_curl_minus_update(g, h->st, aE, aB, nullptr, -hh, 0.f, aE, s), "adjoint: third stage");
    CK(h, launch_grad_minus(g, M, aE, Bh, (double)dt, grad, s), "adjoint: gradient (second stage)");
    if (h->hlen > 0) {
        CK(h, cudaMemcpyAsync(W, aE, sizeof(float) * N, cudaMemcpyDeviceToDevice, s), "adjoint: copy aE1");
        CK(h, launch_correct_j1(g, h->hf, h->hlen, W, s), "adjoint: P^-1 aE1");
        CK(h, launch_grad_corr(g, M, W, J, (double)dt, grad, s), "adjoint: gradient (correction)");
    }
    CK(h, launch_curl_plus_update(g, h->st, aB, aE, dt, aB, s), "adjoint: second stage");
    CK(h, launch_grad_plus(g, M, aB, E, -(double)hh, grad, s), "adjoint: gradient (first stage)");
    CK(h, launch_curl_minus_update(g, h->st, aE, aB, nullptr, -hh, 0.f, aE, s), "adjoint: first stage");
    return PIC_OK;
}

// Tile autotuner: time every field-advance tile variant on this handle's bound fields (the
// output goes to the library's second buffer, so the state is unchanged) and keep the fastest.
// The choice is cached per (ndim, stencil class, nz, nx, ny) for the process.
pic_status pic_autotune(pic_t* h, void* stream) {
    if (!h) return PIC_ERR_ARG;
    pic_status st = need_fields(h);
    if (st) return st;
    if (h->ks) return PIC_OK;           // one k-space advance: nothing to choose
    static std::vector<std::pair<std::vector<long long>, int>> cache;
    const int mclass = h->st.M <= 1 ? 1 : h->st.M <= 4 ? 4 : h->st.M <= 8 ? 8 : 16;
    std::vector<long long> key = {h->g.ndim, mclass, h->g.nz, h->g.nx, h->g.ny};
    for (auto& e : cache)
        if (e.first == key) {
            h->fa_variant = e.second;
            return PIC_OK;
        }
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = h->g.ncell;
    FieldP p;
    p.g = h->g;
    p.st = h->st;
    p.Ein = h->E;
    p.Bin = h->B;
    p.J1 = h->J;
    p.J2 = h->J + N;
    p.J3 = h->J + 2 * N;
    p.Eout = h->E2;
    p.Bout = h->B2;
    p.shift = 0;
    cudaEvent_t a, b;
    CK(h, cudaEventCreate(&a), "event");
    CK(h, cudaEventCreate(&b), "event");
    int best = 0;
    double best_ms = 1e30;
    const int nv = field_variants(h->g.ndim);
    for (int v = 0; v < nv; ++v) {
        cudaError_t e = launch_field_advance(p, s, v);          // warm-up (and attribute set-up)
        for (int r = 0; e == cudaSuccess && r < 2; ++r) e = launch_field_advance(p, s, v);
        if (e == cudaSuccess) e = cudaEventRecord(a, s);
        for (int r = 0; e == cudaSuccess && r < 5; ++r) e = launch_field_advance(p, s, v);
        if (e == cudaSuccess) e = cudaEventRecord(b, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
        if (e != cudaSuccess) {
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            return cuda_fail(h, e, "autotune");
        }
        h->fa_ms[v] = ms / 5.0;
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    h->fa_variant = best;
    cache.push_back({key, best});
    return PIC_OK;
}

pic_status pic_set_tuning(pic_t* h, int variant) {
    if (!h) return PIC_ERR_ARG;
    if (variant < 0 || variant >= field_variants(h->g.ndim)) return fail(h, PIC_ERR_ARG, "tile variant %d", variant);
    h->fa_variant = variant;
    return PIC_OK;
}

pic_status pic_get_tuning(const pic_t* h, int* variant, double* ms, int* nvariants) {
    if (!h) return PIC_ERR_ARG;
    if (variant) *variant = h->fa_variant;
    int nv = field_variants(h->g.ndim);
    if (nvariants) *nvariants = nv;
    if (ms)
        for (int v = 0; v < nv; ++v) ms[v] = h->fa_ms[v];
    return PIC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batched runs ----
struct pic_batch_t {
    std::vector<pic_t*> h;
    // per field-class tables (index: stencil class 0..3 = M <= 1, 4, 8, 16)
    struct FieldGroup {
        std::vector<int> members;
        FieldP* d_inst = nullptr;
        int* d_tiles = nullptr;
        int4* d_work = nullptr;      // 2D: x-marching work items (instance, z0, first row, end row)
        int total = 0, maxm = 1, nwork = 0;
        int variant = 1;             // 0: one cell per thread, 1: register-blocked, 2: x-marching (2D)
        double ms[3] = {0, 0, 0};    // batch autotune: time of one launch per variant (0: not timed)
    } fg[4];
    struct PartGroup {
        std::vector<int> members;
        PartInst* d_inst = nullptr;
        long long max_extent = 0, max_ncell = 0;
        int shape = 1;
    } pg[2];            // shape 1, 2
    CorrInst* d_corr = nullptr;
    int ncorr = 0, max_rows = 0, max_nz = 0;
    FiltInst* d_filt = nullptr;
    int nfilt = 0;
    long long max_rows3 = 0;
    int ndim = 2;
    bool built = false;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t graph = nullptr;       // two steps (one per field-buffer parity)
    cudaGraphExec_t graph_long = nullptr;  // kLongSteps steps, replayed while that many remain
    char err[256] = {0};
};

namespace {

int stencil_class(int M) { return M <= 1 ? 0 : M <= 4 ? 1 : M <= 8 ? 2 : 3; }

template <typename T>
cudaError_t upload(T** d, const std::vector<T>& v) {
    if (*d) cudaFree(*d);
    *d = nullptr;
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void**)d, sizeof(T) * v.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

pic_status bfail(pic_batch_t* b, pic_status st, const char* what) {
    snprintf(b->err, sizeof b->err, "%s", what);
    snprintf(g_create_err, sizeof g_create_err, "%s", what);
    return st;
}

// device tables of a batch (after all instances are bound)
pic_status batch_build(pic_batch_t* b) {
    for (auto& f : b->fg) f.members.clear();
    for (auto& q : b->pg) q.members.clear();
    std::vector<CorrInst> corr;
    std::vector<FiltInst> filt;
    b->max_rows = b->max_nz = 0;
    b->max_rows3 = 0;
    for (int i = 0; i < (int)b->h.size(); ++i) {
        pic_t* h = b->h[i];
        if (!h->E || !h->sp[0].bound) return bfail(b, PIC_ERR_STATE, "batch instance not bound (fields and species 0)");
        b->fg[stencil_class(h->st.M)].members.push_back(i);
        b->pg[h->cfg.shape - 1].members.push_back(i);
        if (h->cfg.current_filter) {
            FiltInst f;
            f.g = h->g;
            f.J = h->J;
            f.vec4 = filter_vec4_ok(h->J, h->g.nz) ? 1 : 0;
            filt.push_back(f);
            b->max_rows3 = std::max(b->max_rows3, 3LL * h->g.nx * h->g.ny);
        }
        if (h->hlen > 0) {
            CorrInst c;
            c.g = h->g;
            c.hlen = h->hlen;
            for (int k = 0; k < 2 * PIC_MAX_HLEN + 1; ++k) {     // centred on PIC_MAX_HLEN
                const int m = k - PIC_MAX_HLEN;
                c.h[k] = (m >= -h->hlen && m <= h->hlen) ? h->hf[m + h->hlen] : 0.f;
            }
            c.J1 = h->J;
            corr.push_back(c);
            long long rows = (long long)h->g.nx * h->g.ny;
            if (rows > b->max_rows) b->max_rows = (int)rows;
            if (h->g.nz > b->max_nz) b->max_nz = h->g.nz;
        }
    }
    static const int maxm_of[4] = {1, 4, 8, 16};
    for (int c = 0; c < 4; ++c) {
        auto& f = b->fg[c];
        std::vector<FieldP> inst;
        std::vector<int> tiles(1, 0);
        std::vector<int4> work;
        for (int j = 0; j < (int)f.members.size(); ++j) {
            pic_t* h = b->h[f.members[j]];
            const bool aligned = ((uintptr_t)h->E | (uintptr_t)h->B | (uintptr_t)h->J | (uintptr_t)h->E2 |
                                  (uintptr_t)h->B2) % 16 == 0;
            for (int par = 0; par < 2; ++par) {
                FieldP p;
                p.g = h->g;
                p.st = h->st;
                p.Ein = par ? h->E2 : h->E;
                p.Bin = par ? h->B2 : h->B;
                p.J1 = h->J;
                p.J2 = h->J + h->g.ncell;
                p.J3 = h->J + 2 * h->g.ncell;
                p.Eout = par ? h->E : h->E2;
                p.Bout = par ? h->B : h->B2;
                p.shift = 0;
                p.vec4 = (h->g.nz % 4 == 0 && aligned) ? 1 : 0;
                inst.push_back(p);
            }
            tiles.push_back(tiles.back() + field_tiles(b->ndim, maxm_of[c], h->g.nz, h->g.nx, h->g.ny));
            if (b->ndim == 2)
                for (int z0 = 0; z0 < h->g.nz; z0 += MARCH2_BATCH_TZ)
                    for (int xa = 0; xa < h->g.nx; xa += MARCH2_BATCH_XC)
                        work.push_back(make_int4(j, z0, xa, std::min(xa + MARCH2_BATCH_XC, h->g.nx)));
        }
        f.total = tiles.back();
        f.maxm = maxm_of[c];
        f.nwork = (int)work.size();
        if (upload(&f.d_inst, inst) != cudaSuccess || upload(&f.d_tiles, tiles) != cudaSuccess ||
            upload(&f.d_work, work) != cudaSuccess)
            return bfail(b, PIC_ERR_OOM, "batch field tables");
    }
    for (int sh = 0; sh < 2; ++sh) {
        auto& q = b->pg[sh];
        std::vector<PartInst> inst;
        q.max_extent = q.max_ncell = 0;
        q.shape = sh + 1;
        for (int i : q.members) {
            pic_t* h = b->h[i];
            PartInst p;
            p.g = h->g;
            p.sp = species_params(h, 0);
            p.E[0] = h->E;
            p.E[1] = h->E2;
            p.B[0] = h->B;
            p.B[1] = h->B2;
            p.J = h->J;
            inst.push_back(p);
            q.max_extent = std::max(q.max_extent, h->sp[0].extent);
            q.max_ncell = std::max(q.max_ncell, h->g.ncell);
        }
        if (upload(&q.d_inst, inst) != cudaSuccess) return bfail(b, PIC_ERR_OOM, "batch particle tables");
    }
    b->ncorr = (int)corr.size();
    if (upload(&b->d_corr, corr) != cudaSuccess) return bfail(b, PIC_ERR_OOM, "batch correction table");
    b->nfilt = (int)filt.size();
    if (upload(&b->d_filt, filt) != cudaSuccess) return bfail(b, PIC_ERR_OOM, "batch filter table");
    b->built = true;
    return PIC_OK;
}

cudaError_t batch_field_launch(pic_batch_t* b, const pic_batch_t::FieldGroup& f, int variant, int parity,
                               cudaStream_t s) {
    const int n = (int)f.members.size();
    if (variant == 2 && b->ndim == 2)
        return launch_field_advance_march2_batch(f.d_inst, f.d_work, f.nwork, f.maxm, parity, s);
    if (variant == 1) return launch_field_advance_rb_batch(f.d_inst, f.d_tiles, n, f.total, b->ndim, f.maxm, parity, s);
    return launch_field_advance_batch(f.d_inst, f.d_tiles, n, f.total, b->ndim, f.maxm, parity, s);
}

// Batch autotune: per stencil class, time one field-advance launch (parity 0: reads E, B, J,
// writes the second buffers, which the step overwrites) with each variant and keep the fastest.
pic_status batch_autotune(pic_batch_t* b, cudaStream_t s) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, PIC_ERR_CUDA, "batch autotune events");
    pic_status st = PIC_OK;
    for (auto& f : b->fg) {
        if (f.members.empty()) continue;
        const int nv = b->ndim == 2 ? 3 : 2;
        double best = 1e30;
        for (int v = 0; v < nv && st == PIC_OK; ++v) {
            cudaError_t e = batch_field_launch(b, f, v, 0, s);            // warm-up
            float ms = 0.f, tot = 0.f;
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
                e = cudaEventRecord(e0, s);
                if (e == cudaSuccess) e = batch_field_launch(b, f, v, 0, s);
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                tot += ms;
            }
            if (e != cudaSuccess) {
                st = bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
                break;
            }
            f.ms[v] = tot / 3.0;
            if (f.ms[v] < best) {
                best = f.ms[v];
                f.variant = v;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

// one step of every instance, reading the field buffers of this parity
cudaError_t batch_enqueue_step(pic_batch_t* b, int parity, cudaStream_t s) {
    cudaError_t e;
    for (auto& q : b->pg)
        if (!q.members.empty() && (e = launch_zero_j_batch(q.d_inst, (int)q.members.size(), q.max_ncell, s))) return e;
    for (auto& q : b->pg)
        if (!q.members.empty() &&
            (e = launch_push_batch(q.d_inst, (int)q.members.size(), b->ndim, q.shape, q.max_extent, parity, s)))
            return e;
    if (b->nfilt && (e = launch_filter_current_batch(b->d_filt, b->nfilt, b->max_rows3, s))) return e;
    if (b->ncorr && (e = launch_correct_j1_batch(b->d_corr, b->ncorr, b->max_rows, b->max_nz, s))) return e;
    for (auto& f : b->fg) {
        if (f.members.empty()) continue;
        if ((e = batch_field_launch(b, f, f.variant, parity, s))) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

pic_status pic_batch_create(const pic_config* cfgs, int n, pic_batch_t** out) {
    if (!cfgs || !out || n < 1) return fail(nullptr, PIC_ERR_ARG, "pic_batch_create: need n >= 1 configs");
    *out = nullptr;
    pic_batch_t* b = new (std::nothrow) pic_batch_t();
    if (!b) return fail(nullptr, PIC_ERR_OOM, "host allocation");
    b->ndim = cfgs[0].ndim;
    for (int i = 0; i < n; ++i) {
        if (cfgs[i].moving_window || cfgs[i].sort_every || cfgs[i].ndim != b->ndim) {
            pic_batch_destroy(b);
            return fail(nullptr, PIC_ERR_ARG, "batch instance %d: same ndim for all, no moving window, no sort", i);
        }
        if (cfgs[i].solver != PIC_SOLVER_YEE && cfgs[i].solver != PIC_SOLVER_CUSTOM) {
            pic_batch_destroy(b);
            return fail(nullptr, PIC_ERR_ARG, "batch instance %d: finite-difference solvers only", i);
        }
        pic_t* h = nullptr;
        pic_status st = pic_create(&cfgs[i], &h);
        if (st) {
            char msg[256];
            snprintf(msg, sizeof msg, "batch instance %d: %s", i, g_create_err);
            snprintf(g_create_err, sizeof g_create_err, "%s", msg);
            pic_batch_destroy(b);
            return st;
        }
        b->h.push_back(h);
    }
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
        pic_batch_destroy(b);
        return fail(nullptr, PIC_ERR_CUDA, "batch capture stream");
    }
    *out = b;
    return PIC_OK;
}

pic_status pic_batch_instance(pic_batch_t* b, int i, pic_t** h) {
    if (!b || !h || i < 0 || i >= (int)b->h.size()) return PIC_ERR_ARG;
    *h = b->h[i];
    b->built = false;            // bindings may change: rebuild tables and graphs at the next step
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->graph_long) {
        cudaGraphExecDestroy(b->graph_long);
        b->graph_long = nullptr;
    }
    return PIC_OK;
}

pic_status pic_batch_step(pic_batch_t* b, int nsteps, void* stream) {
    if (!b || nsteps < 0) return PIC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!b->built) {
        pic_status st = batch_build(b);
        if (!st) st = batch_autotune(b, s);
        if (st) return st;
    }
    // record `steps` (even) steps of every instance into one executable graph
    auto capture = [&](int steps, cudaGraphExec_t* out) -> cudaError_t {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t ek = cudaSuccess;
            for (int k = 0; k < steps && ek == cudaSuccess; ++k) ek = batch_enqueue_step(b, k & 1, b->cap);
            e = cudaStreamEndCapture(b->cap, &g);
            if (e == cudaSuccess) e = ek;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
        if (g) cudaGraphDestroy(g);
        return e;
    };
    if (!b->graph) {
        cudaError_t e = capture(2, &b->graph);
        if (e != cudaSuccess) return bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
    }
    constexpr int kLongSteps = 32;
    int k = 0;
    if (nsteps >= kLongSteps) {
        if (!b->graph_long) {
            cudaError_t e = capture(kLongSteps, &b->graph_long);
            if (e != cudaSuccess) return bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
        }
        for (; k + kLongSteps <= nsteps; k += kLongSteps) {
            cudaError_t e = cudaGraphLaunch(b->graph_long, s);
            if (e != cudaSuccess) return bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    for (; k + 1 < nsteps; k += 2) {
        cudaError_t e = cudaGraphLaunch(b->graph, s);
        if (e != cudaSuccess) return bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
    }
    if (nsteps % 2) {
        cudaError_t e = batch_enqueue_step(b, 0, s);
        for (pic_t* h : b->h) {
            if (e != cudaSuccess) break;
            const size_t bytes = sizeof(float) * 3 * h->g.ncell;
            e = cudaMemcpyAsync(h->E, h->E2, bytes, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->B, h->B2, bytes, cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return bfail(b, PIC_ERR_CUDA, cudaGetErrorString(e));
    }
    for (pic_t* h : b->h) h->step += nsteps;
    return PIC_OK;
}

pic_status pic_batch_get_tuning(const pic_batch_t* b, int* variant, double* ms) {
    if (!b) return PIC_ERR_ARG;
    for (int c = 0; c < 4; ++c) {
        if (variant) variant[c] = b->fg[c].members.empty() ? -1 : b->fg[c].variant;
        if (ms)
            for (int v = 0; v < 3; ++v) ms[3 * c + v] = b->fg[c].ms[v];
    }
    return PIC_OK;
}

pic_status pic_batch_destroy(pic_batch_t* b) {
    if (!b) return PIC_OK;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->graph_long) cudaGraphExecDestroy(b->graph_long);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (auto& f : b->fg) {
        dfree(f.d_inst);
        dfree(f.d_tiles);
        dfree(f.d_work);
    }
    for (auto& q : b->pg) dfree(q.d_inst);
    dfree(b->d_corr);
    dfree(b->d_filt);
    for (pic_t* h : b->h) pic_destroy(h);
    delete b;
    return PIC_OK;
}

}  // extern "C"
