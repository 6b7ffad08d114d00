// C ABI of the GB300 S-model DVM library: context, mesh topology and geometry,
// boundary conditions, initialisation, stepping, moments, checkpoints.
// Declarations and argument conventions: include/dvm.h.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dvm_context.h"

namespace dvm {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

namespace {

// quads of a VTK-ordered hexahedron, outward by the right-hand rule
const int kHexFace[6][4] = {{0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4},
                            {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};

// (1/2)(p2 - p0) x (p3 - p1) and the vertex centroid of a quad
void quad_vec(const double *xyz, const int64_t *v, double A[3], double cen[3]) {
  const double *p0 = xyz + 3 * v[0], *p1 = xyz + 3 * v[1], *p2 = xyz + 3 * v[2],
               *p3 = xyz + 3 * v[3];
  double d1[3], d2[3];
  for (int k = 0; k < 3; ++k) {
    d1[k] = p2[k] - p0[k];
    d2[k] = p3[k] - p1[k];
    cen[k] = 0.25 * ((p0[k] + p1[k]) + (p2[k] + p3[k]));
  }
  A[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
  A[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
  A[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
}

struct FaceKey {
  int64_t k[4];
  int32_t cell;
  int32_t lf;
};

}  // namespace

int build_topology(dvm_ctx *C, const dvm_mesh *m) {
  const int64_t nc = m->n_cell;
  C->slot_nb.assign(6 * nc, -1);
  C->slot_group.assign(6 * nc, -1);
  C->slot_owner.assign(6 * nc, 1);
  C->slot_A.assign(18 * nc, 0.0);
  C->vol.assign(nc, 0.0);
  std::vector<int32_t> bmark(6 * nc, -1);
  for (int64_t b = 0; b < m->n_bface; ++b) {
    const int64_t c = m->bface[2 * b], l = m->bface[2 * b + 1];
    const int32_t g = m->bface_group[b];
    if (c < 0 || c >= nc || l < 0 || l > 5 || g < 0 || g >= kMaxGroups) {
      set_error("boundary face " + std::to_string(b) + " out of range");
      return DVM_ERR_INVALID_ARG;
    }
    if (bmark[6 * c + l] >= 0) {
      set_error("boundary face listed twice");
      return DVM_ERR_INVALID_ARG;
    }
    bmark[6 * c + l] = g;
  }
  std::vector<FaceKey> keys(6 * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int l = 0; l < 6; ++l) {
      FaceKey &k = keys[6 * c + l];
      for (int q = 0; q < 4; ++q) {
        const int64_t v = m->hex8[8 * c + kHexFace[l][q]];
        if (v < 0 || v >= m->n_vert) {
          set_error("vertex id out of range in hex8");
          return DVM_ERR_INVALID_ARG;
        }
        k.k[q] = v;
      }
      std::sort(k.k, k.k + 4);
      k.cell = (int32_t)c;
      k.lf = l;
    }
  std::sort(keys.begin(), keys.end(), [](const FaceKey &a, const FaceKey &b) {
    for (int q = 0; q < 4; ++q)
      if (a.k[q] != b.k[q]) return a.k[q] < b.k[q];
    if (a.cell != b.cell) return a.cell < b.cell;
    return a.lf < b.lf;
  });
  C->face_slot.clear();
  size_t i = 0;
  while (i < keys.size()) {
    size_t j = i + 1;
    while (j < keys.size() && std::equal(keys[j].k, keys[j].k + 4, keys[i].k)) ++j;
    const size_t cnt = j - i;
    if (cnt > 2) {
      set_error("a face is shared by more than two cells");
      return DVM_ERR_INVALID_ARG;
    }
    const int64_t so = 6 * (int64_t)keys[i].cell + keys[i].lf;
    C->face_slot.push_back(so);
    if (cnt == 2) {
      const int64_t sn = 6 * (int64_t)keys[i + 1].cell + keys[i + 1].lf;
      if (bmark[so] >= 0 || bmark[sn] >= 0) {
        set_error("an interior face is listed as a boundary face");
        return DVM_ERR_INVALID_ARG;
      }
      C->slot_nb[so] = keys[i + 1].cell;
      C->slot_nb[sn] = keys[i].cell;
      C->slot_owner[sn] = 0;
      C->face_other.push_back(sn);
    } else {
      if (bmark[so] < 0) {
        set_error("a face without neighbour is not listed as a boundary face");
        return DVM_ERR_INVALID_ARG;
      }
      C->slot_group[so] = bmark[so];
      C->face_other.push_back(-1);
    }
    i = j;
  }
  C->nf = (int64_t)C->face_slot.size();
  // area vectors: the owner's quad defines the face, the neighbour sees its negative
  for (int64_t f = 0; f < C->nf; ++f) {
    const int64_t so = C->face_slot[f];
    const int64_t c = so / 6, l = so % 6;
    int64_t v[4];
    for (int q = 0; q < 4; ++q) v[q] = m->hex8[8 * c + kHexFace[l][q]];
    double A[3], cen[3];
    quad_vec(m->xyz, v, A, cen);
    for (int k = 0; k < 3; ++k) C->slot_A[3 * so + k] = A[k];
    const int64_t sn = C->face_other[f];
    if (sn >= 0)
      for (int k = 0; k < 3; ++k) C->slot_A[3 * sn + k] = -A[k];
  }
  // volumes: divergence theorem over each cell's own quads (exact for trilinear hexes)
  for (int64_t c = 0; c < nc; ++c) {
    double s = 0.0;
    for (int l = 0; l < 6; ++l) {
      int64_t v[4];
      for (int q = 0; q < 4; ++q) v[q] = m->hex8[8 * c + kHexFace[l][q]];
      double A[3], cen[3];
      quad_vec(m->xyz, v, A, cen);
      s += cen[0] * A[0] + cen[1] * A[1] + cen[2] * A[2];
    }
    C->vol[c] = s / 3.0;
    if (!(C->vol[c] > 0.0)) {
      set_error("cell " + std::to_string(c) + " has non-positive volume");
      return DVM_ERR_INVALID_ARG;
    }
  }
  return DVM_OK;
}

}  // namespace dvm

using namespace dvm;

extern "C" {

const char *dvm_last_error(void) { return dvm::g_last_error.c_str(); }

int dvm_create(dvm_ctx **out, const dvm_mesh *mesh, const dvm_vgrid *vg, const dvm_gas *gas,
               const dvm_opts *opts) {
  if (!out || !mesh || !vg || !gas || !opts) {
    set_error("dvm_create: null argument");
    return DVM_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (mesh->n_cell < 1 || mesh->n_cell > 2147483647LL || mesh->n_vert < 8 || !mesh->xyz ||
      !mesh->hex8 || mesh->n_bface < 0 || (mesh->n_bface > 0 && (!mesh->bface || !mesh->bface_group))) {
    set_error("dvm_create: bad mesh sizes or pointers");
    return DVM_ERR_INVALID_ARG;
  }
  for (int a = 0; a < 3; ++a)
    if (vg->N[a] < 2 || vg->N[a] > kMaxN || !(vg->hi[a] > vg->lo[a]) || !std::isfinite(vg->lo[a]) ||
        !std::isfinite(vg->hi[a])) {
      set_error("dvm_create: bad velocity grid");
      return DVM_ERR_INVALID_ARG;
    }
  if (!(gas->Kn > 0.0) || !(gas->Pr > 0.0) || !std::isfinite(gas->omega)) {
    set_error("dvm_create: bad gas parameters");
    return DVM_ERR_INVALID_ARG;
  }
  if (opts->format != DVM_FORMAT_FULL && opts->format != DVM_FORMAT_TUCKER) {
    set_error("dvm_create: unknown format");
    return DVM_ERR_INVALID_ARG;
  }
  if (opts->engine != DVM_ENGINE_AUTO && opts->engine != DVM_ENGINE_CUDA_CORES) {
    set_error("dvm_create: engine must be DVM_ENGINE_AUTO or DVM_ENGINE_CUDA_CORES");
    return DVM_ERR_INVALID_ARG;
  }
  if (opts->scheme != DVM_SCHEME_EXPLICIT && opts->scheme != DVM_SCHEME_LUSGS) {
    set_error("dvm_create: scheme must be DVM_SCHEME_EXPLICIT or DVM_SCHEME_LUSGS");
    return DVM_ERR_INVALID_ARG;
  }
  if (opts->scheme == DVM_SCHEME_LUSGS && opts->format != DVM_FORMAT_FULL) {
    set_error("dvm_create: the LU-SGS scheme is implemented for the full format only");
    return DVM_ERR_UNSUPPORTED;
  }
  if (opts->max_chunk < 0) {
    set_error("dvm_create: max_chunk must be >= 0");
    return DVM_ERR_INVALID_ARG;
  }
  if (opts->variant < DVM_VARIANT_AUTO || opts->variant > DVM_VARIANT_PHASED) {
    set_error("dvm_create: variant must be DVM_VARIANT_AUTO, _FUSED or _PHASED");
    return DVM_ERR_INVALID_ARG;
  }
  if (opts->format == DVM_FORMAT_TUCKER &&
      (opts->rank_cap < 1 || opts->rank_cap > std::min(24, std::min(vg->N[0], std::min(vg->N[1], vg->N[2]))) ||
       !(opts->tol >= 0.0))) {
    set_error("dvm_create: bad Tucker rank cap or tolerance");
    return DVM_ERR_INVALID_ARG;
  }
  dvm_ctx *C = new dvm_ctx();
  C->vg = *vg;
  C->gas = *gas;
  C->opts = *opts;
  if (!(C->opts.cfl > 0.0)) C->opts.cfl = 0.5;
  C->stream = static_cast<cudaStream_t>(opts->cuda_stream);
  C->nc = mesh->n_cell;
  C->nn = 1;
  double m2 = 0.0;
  double dxi[3];
  for (int a = 0; a < 3; ++a) {
    C->N[a] = vg->N[a];
    C->xi[a].resize(vg->N[a]);
    for (int i = 0; i < vg->N[a]; ++i)
      C->xi[a][i] = ((double)(vg->N[a] - 1 - i) * vg->lo[a] + (double)i * vg->hi[a]) /
                    (double)(vg->N[a] - 1);
    dxi[a] = (vg->hi[a] - vg->lo[a]) / (double)(vg->N[a] - 1);
    C->nn *= vg->N[a];
    const double am = std::max(std::fabs(vg->lo[a]), std::fabs(vg->hi[a]));
    m2 += am * am;
  }
  C->w = dxi[0] * dxi[1] * dxi[2];
  C->xi_max = std::sqrt(m2);
  int rc = build_topology(C, mesh);
  if (rc != DVM_OK) {
    delete C;
    return rc;
  }
  C->bc_type.assign(kMaxGroups, -1);
  C->bc_par.assign(kMaxGroups, std::array<double, 8>{});
  if (cudaGetDevice(&C->device) != cudaSuccess) {
    set_error("dvm_create: no CUDA device");
    delete C;
    return DVM_ERR_CUDA;
  }
  rc = ctx_alloc_state(C);
  if (rc != DVM_OK) {
    ctx_free(C);
    delete C;
    return rc;
  }
  *out = C;
  return DVM_OK;
}

int dvm_set_bc(dvm_ctx *C, int32_t group, int32_t type, const double params[8]) {
  if (!C || group < 0 || group >= kMaxGroups || type < DVM_BC_FREESTREAM || type > DVM_BC_WALL) {
    set_error("dvm_set_bc: bad argument");
    return DVM_ERR_INVALID_ARG;
  }
  if (C->initialized) {
    set_error("dvm_set_bc: boundary conditions are fixed after initialisation");
    return DVM_ERR_STATE;
  }
  std::array<double, 8> p{};
  if (params)
    for (int k = 0; k < 8; ++k) p[k] = params[k];
  if (type == DVM_BC_FREESTREAM && !(p[0] > 0.0 && p[4] > 0.0)) {
    set_error("dvm_set_bc: free stream needs n > 0 and T > 0");
    return DVM_ERR_INVALID_ARG;
  }
  if (type == DVM_BC_WALL && !(p[4] > 0.0)) {
    set_error("dvm_set_bc: wall needs T > 0");
    return DVM_ERR_INVALID_ARG;
  }
  C->bc_type[group] = type;
  C->bc_par[group] = p;
  return DVM_OK;
}

int dvm_init_maxwellian(dvm_ctx *C, const double *n, const double *u, const double *T) {
  if (!C || !n || !u || !T) {
    set_error("dvm_init_maxwellian: null argument");
    return DVM_ERR_INVALID_ARG;
  }
  for (int64_t c = 0; c < C->nc; ++c)
    if (!(n[c] > 0.0) || !(T[c] > 0.0) || !std::isfinite(u[3 * c]) || !std::isfinite(u[3 * c + 1]) ||
        !std::isfinite(u[3 * c + 2])) {
      set_error("dvm_init_maxwellian: n and T must be positive and u finite");
      return DVM_ERR_INVALID_ARG;
    }
  int rc = ctx_prepare_boundaries(C);
  if (rc == DVM_OK) rc = ctx_clear_flag(C);
  if (rc != DVM_OK) return rc;
  return ctx_init_from_maxwellians(C, n, u, T);
}

int dvm_init_f(dvm_ctx *C, const double *f, int32_t on_device) {
  if (!C || !f) {
    set_error("dvm_init_f: null argument");
    return DVM_ERR_INVALID_ARG;
  }
  int rc = ctx_prepare_boundaries(C);
  if (rc == DVM_OK) rc = ctx_clear_flag(C);
  if (rc != DVM_OK) return rc;
  return ctx_init_from_full(C, f, on_device != 0);
}

int dvm_init_tucker(dvm_ctx *C, const int32_t *ranks, const double *core, const double *u1,
                    const double *u2, const double *u3, int32_t on_device) {
  if (!C || !ranks || !core || !u1 || !u2 || !u3) {
    set_error("dvm_init_tucker: null argument");
    return DVM_ERR_INVALID_ARG;
  }
  if (C->opts.format != DVM_FORMAT_TUCKER || !C->tucker) {
    set_error("dvm_init_tucker: the context is not in Tucker format");
    return DVM_ERR_INVALID_ARG;
  }
  int rc = ctx_prepare_boundaries(C);
  if (rc == DVM_OK) rc = ctx_clear_flag(C);
  if (rc != DVM_OK) return rc;
  const double *fac[3] = {u1, u2, u3};
  rc = tucker_set_state(C, ranks, core, fac, on_device != 0);
  if (rc == DVM_OK) C->initialized = true;
  return rc;
}

int dvm_get_tucker(dvm_ctx *C, int32_t *ranks, double *core, double *u1, double *u2, double *u3) {
  if (!C) return DVM_ERR_INVALID_ARG;
  if (C->opts.format != DVM_FORMAT_TUCKER || !C->tucker) {
    set_error("dvm_get_tucker: the context is not in Tucker format");
    return DVM_ERR_INVALID_ARG;
  }
  if (!C->initialized) {
    set_error("dvm_get_tucker: context not initialised");
    return DVM_ERR_STATE;
  }
  double *fac[3] = {u1, u2, u3};
  return tucker_get_state(C, ranks, core, fac);
}

int dvm_step(dvm_ctx *C, int32_t nsteps, double *residual_out) {
  if (!C || nsteps < 0) {
    set_error("dvm_step: bad argument");
    return DVM_ERR_INVALID_ARG;
  }
  if (!C->initialized) {
    set_error("dvm_step: context not initialised");
    return DVM_ERR_STATE;
  }
  return ctx_step(C, nsteps, residual_out);
}

int dvm_moments(dvm_ctx *C, double *out) {
  if (!C || !out) {
    set_error("dvm_moments: null argument");
    return DVM_ERR_INVALID_ARG;
  }
  if (!C->initialized) {
    set_error("dvm_moments: context not initialised");
    return DVM_ERR_STATE;
  }
  return ctx_moments(C, out);
}

int dvm_solve(dvm_ctx *C, double tol, int64_t max_steps, int32_t check_every, int64_t *steps_out,
              double *res_out) {
  if (!C || max_steps < 0 || check_every < 1) {
    set_error("dvm_solve: bad argument");
    return DVM_ERR_INVALID_ARG;
  }
  if (!C->initialized) {
    set_error("dvm_solve: context not initialised");
    return DVM_ERR_STATE;
  }
  int64_t done = 0;
  double res = INFINITY;
  while (done < max_steps) {
    const int32_t k = (int32_t)std::min<int64_t>(check_every, max_steps - done);
    int rc = ctx_step(C, k, &res);
    if (rc != DVM_OK) return rc;
    done += k;
    if (res <= tol) break;
  }
  if (steps_out) *steps_out = done;
  if (res_out) *res_out = res;
  return res <= tol ? DVM_OK : DVM_NOT_CONVERGED;
}

int dvm_get_f(dvm_ctx *C, int64_t cell0, int64_t ncell, double *out) {
  if (!C || !out || cell0 < 0 || ncell < 0 || cell0 + ncell > C->nc) {
    set_error("dvm_get_f: bad range");
    return DVM_ERR_INVALID_ARG;
  }
  if (!C->initialized) {
    set_error("dvm_get_f: context not initialised");
    return DVM_ERR_STATE;
  }
  return ctx_get_f(C, cell0, ncell, out);
}

int dvm_get_dt(dvm_ctx *C, double *dt) {
  if (!C || !dt) return DVM_ERR_INVALID_ARG;
  if (!C->initialized) {
    set_error("dvm_get_dt: context not initialised");
    return DVM_ERR_STATE;
  }
  *dt = C->dt;
  return DVM_OK;
}

int dvm_get_step_count(dvm_ctx *C, int64_t *steps) {
  if (!C || !steps) return DVM_ERR_INVALID_ARG;
  *steps = C->steps;
  return DVM_OK;
}

int dvm_get_num_faces(dvm_ctx *C, int64_t *n_face) {
  if (!C || !n_face) return DVM_ERR_INVALID_ARG;
  *n_face = C->nf;
  return DVM_OK;
}

int dvm_get_geometry(dvm_ctx *C, double *vol, int64_t *fcell, double *fgeo) {
  if (!C) return DVM_ERR_INVALID_ARG;
  if (vol)
    for (int64_t c = 0; c < C->nc; ++c) vol[c] = C->vol[c];
  for (int64_t f = 0; f < C->nf; ++f) {
    const int64_t so = C->face_slot[f];
    const double *A = &C->slot_A[3 * so];
    const double a = std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    if (fcell) {
      fcell[3 * f] = so / 6;
      fcell[3 * f + 1] = C->slot_nb[so];
      fcell[3 * f + 2] = C->slot_group[so];
    }
    if (fgeo) {
      fgeo[4 * f] = a;
      for (int k = 0; k < 3; ++k) fgeo[4 * f + 1 + k] = A[k] / a;
    }
  }
  return DVM_OK;
}

int dvm_get_ranks(dvm_ctx *C, int32_t *r) {
  if (!C || !r) return DVM_ERR_INVALID_ARG;
  return ctx_get_ranks(C, r);
}

int dvm_get_launch_config(dvm_ctx *C, int32_t *grid, float *tune_ms) {
  if (!C) return DVM_ERR_INVALID_ARG;
  if (C->opts.format == DVM_FORMAT_TUCKER && C->tucker) return tucker_launch_info(C, grid, tune_ms);
  if (grid) *grid = (int32_t)C->nc;
  if (tune_ms)
    for (int i = 0; i < 5; ++i) tune_ms[i] = 0.f;
  return DVM_OK;
}

int dvm_set_kernel_timing(dvm_ctx *C, int32_t on) {
  if (!C) return DVM_ERR_INVALID_ARG;
  int rc = ctx_collect_timing(C);
  if (rc != DVM_OK) return rc;
  for (int k = 0; k < kKClasses; ++k) {
    C->timing.ms[k] = 0.0;
    C->timing.launches[k] = 0;
  }
  C->timing.on = on != 0;
  return DVM_OK;
}

int dvm_get_kernel_timing(dvm_ctx *C, double *ms, int64_t *launches) {
  if (!C) return DVM_ERR_INVALID_ARG;
  int rc = ctx_collect_timing(C);
  if (rc != DVM_OK) return rc;
  for (int k = 0; k < kKClasses; ++k) {
    if (ms) ms[k] = C->timing.ms[k];
    if (launches) launches[k] = C->timing.launches[k];
  }
  return DVM_OK;
}

int dvm_memory(dvm_ctx *C, size_t *f_bytes, size_t *total_bytes) {
  if (!C) return DVM_ERR_INVALID_ARG;
  return ctx_memory(C, f_bytes, total_bytes);
}

int dvm_save(dvm_ctx *C, const char *path) {
  if (!C || !path) return DVM_ERR_INVALID_ARG;
  if (!C->initialized) {
    set_error("dvm_save: context not initialised");
    return DVM_ERR_STATE;
  }
  return ctx_save(C, path);
}

int dvm_load(dvm_ctx *C, const char *path) {
  if (!C || !path) return DVM_ERR_INVALID_ARG;
  int rc = ctx_prepare_boundaries(C);
  if (rc == DVM_OK) rc = ctx_clear_flag(C);
  if (rc != DVM_OK) return rc;
  return ctx_load(C, path);
}

void dvm_destroy(dvm_ctx *C) {
  if (!C) return;
  ctx_free(C);
  delete C;
}

int dvm_lusgs_wavefronts(int64_t n_cell, const int32_t *nb, int32_t forward, int32_t *order,
                         int64_t *offsets, int64_t *n_waves) {
  if (n_cell < 0 || n_cell > INT32_MAX || (n_cell > 0 && (!nb || !order)) || !offsets || !n_waves) {
    set_error("dvm_lusgs_wavefronts: bad arguments");
    return DVM_ERR_INVALID_ARG;
  }
  for (int64_t k = 0; k < 6 * n_cell; ++k)
    if (nb[k] < -1 || nb[k] >= n_cell) {
      set_error("dvm_lusgs_wavefronts: neighbour index out of range");
      return DVM_ERR_INVALID_ARG;
    }
  std::vector<int64_t> off;
  lusgs_wavefronts(n_cell, nb, forward != 0, order, off);
  for (size_t w = 0; w < off.size(); ++w) offsets[w] = off[w];
  *n_waves = (int64_t)off.size() - 1;
  return DVM_OK;
}

}  // extern "C"
