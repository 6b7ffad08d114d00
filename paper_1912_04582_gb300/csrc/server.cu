// Serving: continuous batching of steady-state S-model solves on one GPU.
//
// Requests wait in a FIFO queue until a slot is free and their device-memory
// estimate fits in what the running solves leave of the budget.  Each admitted
// request gets its own context on its own CUDA stream.  The loop keeps every
// running solve in flight: it enqueues `check_every` steps plus an
// asynchronous residual read-back, records an event, and services whichever
// solves have completed (cudaEventQuery) — a small, fast solve iterates many
// times while a large one works through one chunk, and newly admitted requests
// join as soon as memory frees up.  Finished solves keep their macroparameters
// on the host and release all device memory.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "dvm_context.h"
#include "tucker.h"

using namespace dvm;

int ctx_enqueue_residual(dvm_ctx *C, double *pinned_out);

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int64_t ticket = 0;
  int32_t state = DVM_REQ_QUEUED;
  std::vector<double> xyz, bc_params, n0, u0, T0;
  std::vector<int64_t> hex8, bface;
  std::vector<int32_t> bgroup, bc_group, bc_type;
  int64_t n_vert = 0, n_cell = 0, n_bface = 0;
  dvm_vgrid vg{};
  dvm_gas gas{};
  dvm_opts opts{};
  double tol = 0.0;
  int64_t max_steps = 0;
  int32_t check_every = 1;
  size_t est = 0;
  dvm_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  double *h_out = nullptr;  // pinned: residual, flag
  bool in_flight = false;
  bool cancel = false;  // retire at the end of the chunk in flight
  int64_t steps = 0;
  double res = INFINITY;
  double t_submit = 0.0, t_done = 0.0;
  std::vector<double> macro;
  std::string error;  // message of the failure, if any
};

size_t estimate(const dvm_request *q) {
  const int64_t nc = q->mesh.n_cell;
  int64_t nn = 1, sumN = 0, Nmax = 0;
  for (int a = 0; a < 3; ++a) {
    nn *= q->vgrid.N[a];
    sumN += q->vgrid.N[a];
    Nmax = std::max<int64_t>(Nmax, q->vgrid.N[a]);
  }
  int nghost = 0;
  for (int i = 0; i < q->n_bc; ++i)
    if (q->bc_type[i] == DVM_BC_FREESTREAM || q->bc_type[i] == DVM_BC_WALL) ++nghost;
  size_t b = sizeof(double) * (size_t)(sumN + nc * (1 + 2 * kSums + 3 + 2 + 8)) +
             sizeof(SlotDev) * 6 * (size_t)nc + sizeof(double) * (size_t)nghost * nn;
  if (q->opts.format == DVM_FORMAT_FULL) {
    b += 2 * sizeof(double) * (size_t)nc * nn;
    // implicit step: 1/D~ at every node, per-cell dt nu, the two sweeps' cell lists
    if (q->opts.scheme == DVM_SCHEME_LUSGS)
      b += sizeof(double) * (size_t)nc * (nn + 1) + sizeof(int32_t) * 2 * (size_t)nc;
  } else {
    const int64_t R = q->opts.rank_cap;
    b += 2 * (sizeof(double) * (size_t)nc * (R * R * R + sumN * R) + sizeof(int) * 3 * nc);
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    const size_t es = q->opts.precision == DVM_PREC_FP64 ? 8 : 4;
    const size_t grid = std::min<size_t>((size_t)nc, (size_t)sms * 4);
    b += grid * es * (tucker_scratch_elems(q->vgrid.N[0], q->vgrid.N[1], q->vgrid.N[2], (int)R) + 64);
    b += sizeof(double) * (size_t)nc + sizeof(double) * (size_t)(nghost + 1) * 3 * Nmax;
    // work buffers of the phase-major step variant, if the autotuner keeps it
    b += (size_t)nc * (tucker_split_bytes_per_cell(q->vgrid.N[0], q->vgrid.N[1], q->vgrid.N[2],
                                                   (int)R, (int)Nmax, es == 8) + 64);
    b += (size_t)nc * tucker_split_t2all_bytes_per_cell(q->vgrid.N[0], q->vgrid.N[1],
                                                        q->vgrid.N[2], (int)R, es == 8) + 512;
  }
  return b + b / 20 + (16u << 20);
}

}  // namespace

struct dvm_server {
  size_t budget = 0, used = 0;
  int32_t max_slots = 1;
  int device = 0;
  int64_t next_ticket = 1;
  std::deque<int64_t> queue;
  std::vector<int64_t> running;
  std::map<int64_t, Request> reqs;
};

namespace {

void release(Request &r, dvm_server *S) {
  if (r.ctx) {
    dvm_destroy(r.ctx);
    r.ctx = nullptr;
  }
  if (r.ev) cudaEventDestroy(r.ev);
  if (r.stream) cudaStreamDestroy(r.stream);
  if (r.h_out) cudaFreeHost(r.h_out);
  r.ev = nullptr;
  r.stream = nullptr;
  r.h_out = nullptr;
  S->used -= r.est;
}

// create, set up and initialise the context of an admitted request
int start(Request &r) {
  if (cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost(&r.h_out, 4 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    set_error("server: stream / event / pinned buffer creation failed");
    return DVM_ERR_CUDA;
  }
  dvm_mesh m{r.n_vert, r.xyz.data(), r.n_cell, r.hex8.data(), r.n_bface,
             r.bface.empty() ? nullptr : r.bface.data(), r.bgroup.empty() ? nullptr : r.bgroup.data()};
  dvm_opts o = r.opts;
  o.cuda_stream = r.stream;
  int rc = dvm_create(&r.ctx, &m, &r.vg, &r.gas, &o);
  if (rc != DVM_OK) return rc;
  for (size_t i = 0; i < r.bc_group.size(); ++i) {
    rc = dvm_set_bc(r.ctx, r.bc_group[i], r.bc_type[i], r.bc_params.data() + 8 * i);
    if (rc != DVM_OK) return rc;
  }
  return dvm_init_maxwellian(r.ctx, r.n0.data(), r.u0.data(), r.T0.data());
}

void finish(Request &r, dvm_server *S, int32_t state) {
  r.state = state;
  if (state == DVM_REQ_FAILED && r.error.empty()) r.error = dvm_last_error();
  r.t_done = now_s();
  if (r.ctx && state != DVM_REQ_FAILED) {
    r.macro.resize(8 * (size_t)r.n_cell);
    if (dvm_moments(r.ctx, r.macro.data()) != DVM_OK) r.macro.clear();
  }
  release(r, S);
}

// enqueue the next chunk of steps and the residual read-back
int launch_chunk(Request &r) {
  const int64_t left = r.max_steps - r.steps;
  const int32_t k = (int32_t)std::min<int64_t>(r.check_every, left);
  int rc = dvm_step(r.ctx, k, nullptr);
  if (rc != DVM_OK) return rc;
  r.steps += k;
  r.h_out[1] = 0.0;  // the non-physical flag lands in the low bytes of this slot
  rc = ctx_enqueue_residual(r.ctx, r.h_out);
  if (rc != DVM_OK) return rc;
  if (cudaEventRecord(r.ev, r.stream) != cudaSuccess) return DVM_ERR_CUDA;
  r.in_flight = true;
  return DVM_OK;
}

}  // namespace

extern "C" {

int dvm_estimate_memory(const dvm_request *req, size_t *bytes) {
  if (!req || !bytes || req->mesh.n_cell < 1) {
    set_error("dvm_estimate_memory: bad argument");
    return DVM_ERR_INVALID_ARG;
  }
  *bytes = estimate(req);
  return DVM_OK;
}

int dvm_server_create(dvm_server **out, size_t hbm_budget, int32_t max_slots) {
  if (!out || max_slots < 1 || hbm_budget == 0) {
    set_error("dvm_server_create: bad argument");
    return DVM_ERR_INVALID_ARG;
  }
  dvm_server *S = new dvm_server();
  S->budget = hbm_budget;
  S->max_slots = max_slots;
  cudaGetDevice(&S->device);
  *out = S;
  return DVM_OK;
}

int dvm_server_submit(dvm_server *S, const dvm_request *q, int64_t *ticket) {
  if (!S || !q || !ticket || q->mesh.n_cell < 1 || !q->mesh.xyz || !q->mesh.hex8 || !q->n0 ||
      !q->u0 || !q->T0 || q->n_bc < 0 || (q->n_bc > 0 && (!q->bc_group || !q->bc_type || !q->bc_params)) ||
      q->check_every < 1 || q->max_steps < 1) {
    set_error("dvm_server_submit: bad request");
    return DVM_ERR_INVALID_ARG;
  }
  Request r;
  r.est = estimate(q);
  if (r.est > S->budget) {
    set_error("dvm_server_submit: request needs more device memory than the whole budget");
    return DVM_ERR_INVALID_ARG;
  }
  r.ticket = S->next_ticket++;
  r.n_vert = q->mesh.n_vert;
  r.n_cell = q->mesh.n_cell;
  r.n_bface = q->mesh.n_bface;
  r.xyz.assign(q->mesh.xyz, q->mesh.xyz + 3 * r.n_vert);
  r.hex8.assign(q->mesh.hex8, q->mesh.hex8 + 8 * r.n_cell);
  if (r.n_bface > 0) {
    r.bface.assign(q->mesh.bface, q->mesh.bface + 2 * r.n_bface);
    r.bgroup.assign(q->mesh.bface_group, q->mesh.bface_group + r.n_bface);
  }
  r.vg = q->vgrid;
  r.gas = q->gas;
  r.opts = q->opts;
  r.bc_group.assign(q->bc_group, q->bc_group + q->n_bc);
  r.bc_type.assign(q->bc_type, q->bc_type + q->n_bc);
  r.bc_params.assign(q->bc_params, q->bc_params + 8 * q->n_bc);
  r.n0.assign(q->n0, q->n0 + r.n_cell);
  r.u0.assign(q->u0, q->u0 + 3 * r.n_cell);
  r.T0.assign(q->T0, q->T0 + r.n_cell);
  r.tol = q->tol;
  r.max_steps = q->max_steps;
  r.check_every = q->check_every;
  r.t_submit = now_s();
  *ticket = r.ticket;
  S->queue.push_back(r.ticket);
  S->reqs.emplace(r.ticket, std::move(r));
  return DVM_OK;
}

int dvm_server_run(dvm_server *S, double max_seconds, int64_t *pending) {
  if (!S) return DVM_ERR_INVALID_ARG;
  cudaSetDevice(S->device);
  const double t0 = now_s();
  while (true) {
    // admission: FIFO while a slot is free and the estimate fits
    while (!S->queue.empty() && (int32_t)S->running.size() < S->max_slots) {
      Request &r = S->reqs[S->queue.front()];
      if (S->used + r.est > S->budget || fault_admit()) break;
      S->queue.pop_front();
      S->used += r.est;
      int rc = start(r);
      if (rc != DVM_OK || launch_chunk(r) != DVM_OK) {
        finish(r, S, DVM_REQ_FAILED);
        continue;
      }
      r.state = DVM_REQ_RUNNING;
      S->running.push_back(r.ticket);
    }
    if (S->running.empty() && S->queue.empty()) break;
    // service the solves whose chunk has completed
    bool any = false;
    for (size_t i = 0; i < S->running.size();) {
      Request &r = S->reqs[S->running[i]];
      const cudaError_t q = cudaEventQuery(r.ev);
      if (q == cudaErrorNotReady) {
        ++i;
        continue;
      }
      any = true;
      r.in_flight = false;
      int32_t done = -1;
      if (q != cudaSuccess) {
        cudaGetLastError();
        r.error = std::string("device error: ") + cudaGetErrorString(q);
        done = DVM_REQ_FAILED;
      } else {
        r.res = r.h_out[0];
        int flag = 0;
        std::memcpy(&flag, r.h_out + 1, sizeof flag);
        if (flag != 0 || !std::isfinite(r.res)) {
          r.error = (flag & 2) ? "a bulk shared-memory copy did not complete within its wait "
                                 "limit: the solve's state is undefined"
                    : (flag & 1) ? "non-physical state: n <= 0 or T <= 0 in some cell"
                                 : "residual is not finite";
          done = DVM_REQ_FAILED;
        }
        else if (r.res <= r.tol) done = DVM_REQ_CONVERGED;
        else if (r.cancel) done = DVM_REQ_CANCELLED;
        else if (r.steps >= r.max_steps) done = DVM_REQ_NOT_CONVERGED;
        else if (launch_chunk(r) != DVM_OK) done = DVM_REQ_FAILED;
      }
      if (done >= 0) {
        finish(r, S, done);
        S->running.erase(S->running.begin() + i);
      } else {
        ++i;
      }
    }
    if (now_s() - t0 > max_seconds) break;
    if (!any) std::this_thread::yield();
  }
  if (pending) *pending = (int64_t)(S->queue.size() + S->running.size());
  return DVM_OK;
}

int dvm_server_poll(dvm_server *S, int64_t ticket, int32_t *state, int64_t *steps,
                    double *residual, double *latency_s) {
  if (!S) return DVM_ERR_INVALID_ARG;
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("dvm_server_poll: unknown ticket");
    return DVM_ERR_INVALID_ARG;
  }
  const Request &r = it->second;
  if (state) *state = r.state;
  if (steps) *steps = r.steps;
  if (residual) *residual = r.res;
  if (latency_s) *latency_s = r.t_done > 0.0 ? r.t_done - r.t_submit : 0.0;
  return DVM_OK;
}

int dvm_server_result(dvm_server *S, int64_t ticket, double *macro) {
  if (!S || !macro) return DVM_ERR_INVALID_ARG;
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end() || it->second.macro.empty()) {
    set_error("dvm_server_result: no result for this ticket");
    return DVM_ERR_STATE;
  }
  std::memcpy(macro, it->second.macro.data(), sizeof(double) * it->second.macro.size());
  return DVM_OK;
}

int dvm_server_cancel(dvm_server *S, int64_t ticket) {
  if (!S) return DVM_ERR_INVALID_ARG;
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("dvm_server_cancel: unknown ticket");
    return DVM_ERR_INVALID_ARG;
  }
  Request &r = it->second;
  if (r.state == DVM_REQ_QUEUED) {  // never admitted: nothing on the device
    for (auto q = S->queue.begin(); q != S->queue.end(); ++q)
      if (*q == ticket) {
        S->queue.erase(q);
        break;
      }
    r.state = DVM_REQ_CANCELLED;
    r.t_done = now_s();
    return DVM_OK;
  }
  if (r.state == DVM_REQ_RUNNING) {  // retired by dvm_server_run after its current chunk
    r.cancel = true;
    return DVM_OK;
  }
  set_error("dvm_server_cancel: the request has already finished");
  return DVM_ERR_STATE;
}

const char *dvm_server_error(dvm_server *S, int64_t ticket) {
  if (!S) return "";
  auto it = S->reqs.find(ticket);
  return it == S->reqs.end() ? "unknown ticket" : it->second.error.c_str();
}

void dvm_server_destroy(dvm_server *S) {
  if (!S) return;
  for (int64_t t : S->running) {
    Request &r = S->reqs[t];
    if (r.stream) cudaStreamSynchronize(r.stream);
    release(r, S);
  }
  delete S;
}

}  // extern "C"
