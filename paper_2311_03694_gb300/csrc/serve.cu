// Serving loop: continuous batching of ROM trajectory requests.
//
// Each model (a resident ROM) owns a pool of slots, one grom_traj of
// max_slots trajectories whose `active` mask and per-slot step budget the
// batched kernels honour.  Models run independently: the host loop polls
// each model and, whenever a model's previous quantum has finished,
//   1. retires its finished slots (final state to the host, slot and memory
//      released),
//   2. admits queued requests of that model into free slots while the HBM
//      budget allows (one batched kernel initialises the new slots),
//   3. enqueues its next quantum of steps on its own stream (models created
//      on different streams overlap on the device) followed by a read-back
//      of the step budgets and an event.
// Arrived requests wait in per-model FIFO queues.  The same scheduler runs
// in a simulation mode without a GPU, where a quantum of a model costs
// quantum * step_seconds of virtual time (discrete-event clock).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <new>
#include <thread>
#include <vector>

#include "grom_internal.h"

namespace grom {

struct ServerModel {
  grom_rom* rom = nullptr;  // null in simulation
  int n = 0;
  int slots = 0;
  int64_t rom_bytes = 0;
  double step_seconds = 0.0;  // simulation only
  grom_traj* traj = nullptr;
  std::vector<int> slot_req;  // request index per slot, -1 free
  std::vector<int> free_slots;
  std::deque<int> ready;
  // pinned staging
  int32_t* h_slots = nullptr;
  int32_t* h_horizons = nullptr;
  double* h_u0 = nullptr;
  int32_t* h_left = nullptr;
  int64_t* h_taken = nullptr;
  int32_t* d_slots = nullptr;
  int32_t* d_horizons = nullptr;
  double* d_u0 = nullptr;
  std::vector<int32_t> sim_left;  // simulation: remaining steps per slot
  cudaEvent_t done_ev = nullptr;
  bool in_flight = false;         // a quantum is running
  double sim_done = 0.0;          // simulation: virtual time the quantum ends
};

static int64_t slot_bytes(int n) { return 8 * (7 * (int64_t)n + 4); }

}  // namespace grom

struct grom_server {
  int64_t budget = 0;
  int quantum = 16;
  bool simulate = false;
  int64_t resident = 0;  // charged model bytes
  std::vector<grom::ServerModel> models;
};

using namespace grom;

static void model_free(ServerModel& m) {
  if (m.traj) grom_traj_destroy(m.traj);
  if (m.h_slots) cudaFreeHost(m.h_slots);
  if (m.h_horizons) cudaFreeHost(m.h_horizons);
  if (m.h_u0) cudaFreeHost(m.h_u0);
  if (m.h_left) cudaFreeHost(m.h_left);
  if (m.h_taken) cudaFreeHost(m.h_taken);
  if (m.d_slots) cudaFree(m.d_slots);
  if (m.d_horizons) cudaFree(m.d_horizons);
  if (m.d_u0) cudaFree(m.d_u0);
  if (m.done_ev) cudaEventDestroy(m.done_ev);
  m = ServerModel();
}

extern "C" {

grom_status grom_server_create(int64_t hbm_budget_bytes, int32_t quantum_steps, int32_t simulate, grom_server** out) {
  if (!out) return fail(GROM_ERR_INVALID_ARG, "grom_server_create: null out");
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || quantum_steps < 1)
    return fail(GROM_ERR_INVALID_ARG, "grom_server_create: need a positive budget and quantum");
  grom_server* s = new (std::nothrow) grom_server();
  if (!s) return fail(GROM_ERR_OOM, "grom_server_create: host allocation");
  s->budget = hbm_budget_bytes;
  s->quantum = quantum_steps;
  s->simulate = simulate != 0;
  *out = s;
  return GROM_OK;
}

grom_status grom_server_destroy(grom_server* s) {
  if (!s) return GROM_OK;
  for (auto& m : s->models) model_free(m);
  delete s;
  return GROM_OK;
}

static grom_status add_model(grom_server* s, ServerModel&& m, int32_t* id) {
  const int64_t charge = m.rom_bytes + (int64_t)m.slots * slot_bytes(m.n);
  if (s->resident + charge > s->budget) return fail(GROM_ERR_BUDGET, "model does not fit the HBM budget");
  s->resident += charge;
  m.slot_req.assign(m.slots, -1);
  for (int q = m.slots - 1; q >= 0; --q) m.free_slots.push_back(q);
  s->models.push_back(std::move(m));
  if (id) *id = (int32_t)s->models.size() - 1;
  return GROM_OK;
}

grom_status grom_server_add_simulated(grom_server* s, int32_t n, int64_t rom_bytes, int32_t max_slots,
                                      double step_seconds, int32_t* model) {
  if (!s || !s->simulate) return fail(GROM_ERR_INVALID_ARG, "grom_server_add_simulated: not a simulation server");
  if (n < 1 || max_slots < 1 || rom_bytes < 0 || !(step_seconds >= 0.0))
    return fail(GROM_ERR_INVALID_ARG, "grom_server_add_simulated: bad arguments");
  ServerModel m;
  m.n = n;
  m.slots = max_slots;
  m.rom_bytes = rom_bytes;
  m.step_seconds = step_seconds;
  m.sim_left.assign(max_slots, 0);
  return add_model(s, std::move(m), model);
}

grom_status grom_server_add_rom(grom_server* s, grom_rom* rom, int32_t max_slots, int32_t* model) {
  if (!s || !rom) return fail(GROM_ERR_INVALID_ARG, "grom_server_add_rom: null argument");
  if (s->simulate) return fail(GROM_ERR_INVALID_ARG, "grom_server_add_rom: simulation server");
  if (max_slots < 1 || max_slots > rom->max_batch)
    return fail(GROM_ERR_INVALID_ARG, "grom_server_add_rom: max_slots must be in 1..max_batch of the ROM");
  ServerModel m;
  m.rom = rom;
  m.n = rom->n;
  m.slots = max_slots;
  m.rom_bytes = (int64_t)rom->total_bytes;
  const int64_t charge = m.rom_bytes + (int64_t)m.slots * slot_bytes(m.n);
  if (s->resident + charge > s->budget) return fail(GROM_ERR_BUDGET, "model does not fit the HBM budget");
  // slot pool: zero states, all slots inactive
  std::vector<double> zeros((size_t)max_slots * m.n, 0.0);
  grom_status st = grom_traj_create(rom, max_slots, zeros.data(), &m.traj);
  if (st) return st;
  auto bail = [&](grom_status code) {
    model_free(m);
    return code;
  };
  const size_t nslot = (size_t)max_slots;
  if (cudaMalloc(&m.traj->active, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&m.traj->steps_left, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMemsetAsync(m.traj->active, 0, nslot * sizeof(int32_t), rom->stream) != cudaSuccess ||
      cudaMemsetAsync(m.traj->steps_left, 0, nslot * sizeof(int32_t), rom->stream) != cudaSuccess ||
      cudaMallocHost(&m.h_slots, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&m.h_horizons, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&m.h_u0, nslot * m.n * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&m.h_left, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&m.h_taken, nslot * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&m.d_slots, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&m.d_horizons, nslot * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&m.d_u0, nslot * m.n * sizeof(double)) != cudaSuccess ||
      cudaEventCreateWithFlags(&m.done_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamSynchronize(rom->stream) != cudaSuccess) {
    cudaError_t e = cudaGetLastError();
    return bail(cuda_fail(e == cudaSuccess ? cudaErrorMemoryAllocation : e, "grom_server_add_rom"));
  }
  return add_model(s, std::move(m), model);
}

grom_status grom_serve(grom_server* s, const grom_request* reqs, int32_t count, grom_result* results,
                       grom_serve_stats* stats) {
  TraceRange trace("grom_serve");
  if (!s || (count > 0 && (!reqs || !results))) return fail(GROM_ERR_INVALID_ARG, "grom_serve: null argument");
  const int M = (int)s->models.size();
  for (int32_t q = 0; q < count; ++q) {
    if (reqs[q].model < 0 || reqs[q].model >= M || reqs[q].horizon < 1 || !reqs[q].u0 ||
        !(reqs[q].arrival >= 0.0))
      return fail(GROM_ERR_INVALID_ARG, "grom_serve: bad request " + std::to_string(q));
    results[q] = grom_result{GROM_OK, 0, -1.0, -1.0};
  }
  std::vector<int> order((size_t)count);
  for (int q = 0; q < count; ++q) order[q] = q;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return reqs[a].arrival < reqs[b].arrival; });
  for (auto& m : s->models) {
    m.ready.clear();
    std::fill(m.slot_req.begin(), m.slot_req.end(), -1);
    m.free_slots.clear();
    for (int q = m.slots - 1; q >= 0; --q) m.free_slots.push_back(q);
  }
  const auto wall0 = std::chrono::steady_clock::now();
  double vclock = 0.0;  // simulation time
  auto now = [&]() {
    if (s->simulate) return vclock;
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - wall0).count();
  };
  int64_t used = s->resident, peak_bytes = used, tsteps = 0, quanta = 0;
  int32_t peak_active = 0, active_total = 0, finished = 0;
  size_t next = 0;
  for (auto& m : s->models) m.in_flight = false;

  // Retires the finished slots of model m (its quantum has completed).
  auto retire = [&](ServerModel& m) -> grom_status {
    std::vector<int> done;
    for (int b = 0; b < m.slots; ++b) {
      const int q = m.slot_req[b];
      if (q < 0) continue;
      const int left = s->simulate ? m.sim_left[b] : m.h_left[b];
      if (left <= 0) done.push_back(b);
    }
    if (done.empty()) return GROM_OK;
    if (!s->simulate) {
      for (size_t d = 0; d < done.size(); ++d) {
        const int b = done[d];
        const int q = m.slot_req[b];
        const int64_t l = m.h_taken[b];
        const double* src = m.traj->hist + (int64_t)b * 6 * m.n + (l % 3) * m.n;
        double* dst = reqs[q].u_final ? reqs[q].u_final : m.h_u0 + d * m.n;
        GROM_CUDA_TRY(
            cudaMemcpyAsync(dst, src, (size_t)m.n * sizeof(double), cudaMemcpyDeviceToHost, m.rom->stream));
      }
      GROM_CUDA_TRY(cudaStreamSynchronize(m.rom->stream));
    }
    const double tdone = now();
    for (size_t d = 0; d < done.size(); ++d) {
      const int b = done[d];
      const int q = m.slot_req[b];
      int status = GROM_OK;
      if (!s->simulate) {
        const double* dst = reqs[q].u_final ? reqs[q].u_final : m.h_u0 + d * m.n;
        for (int i = 0; i < m.n; ++i)
          if (!std::isfinite(dst[i])) {
            status = GROM_ERR_NONFINITE;
            break;
          }
        results[q].steps = (int32_t)m.h_taken[b];
      } else {
        results[q].steps = reqs[q].horizon;
      }
      results[q].status = status;
      results[q].t_done = tdone;
      tsteps += reqs[q].horizon;
      m.slot_req[b] = -1;
      m.free_slots.push_back(b);
      used -= slot_bytes(m.n);
      --active_total;
      ++finished;
    }
    return GROM_OK;
  };

  // Admits queued requests of model m into free slots (budget permitting).
  auto admit = [&](ServerModel& m, double t) -> grom_status {
    int nadmit = 0;
    while (!m.ready.empty() && !m.free_slots.empty()) {
      const int q = m.ready.front();
      const int64_t fp = slot_bytes(m.n);
      if (s->resident + fp > s->budget) {  // can never fit
        m.ready.pop_front();
        results[q].status = GROM_ERR_BUDGET;
        results[q].t_admit = results[q].t_done = t;
        ++finished;
        continue;
      }
      if (used + fp > s->budget) break;
      m.ready.pop_front();
      const int slot = m.free_slots.back();
      m.free_slots.pop_back();
      m.slot_req[slot] = q;
      used += fp;
      results[q].t_admit = t;
      ++active_total;
      if (s->simulate) {
        m.sim_left[slot] = reqs[q].horizon;
      } else {
        m.h_slots[nadmit] = slot;
        m.h_horizons[nadmit] = reqs[q].horizon;
        std::memcpy(m.h_u0 + (size_t)nadmit * m.n, reqs[q].u0, (size_t)m.n * sizeof(double));
      }
      ++nadmit;
    }
    if (nadmit > 0 && !s->simulate) {
      cudaStream_t st = m.rom->stream;
      GROM_CUDA_TRY(cudaMemcpyAsync(m.d_slots, m.h_slots, nadmit * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      GROM_CUDA_TRY(
          cudaMemcpyAsync(m.d_horizons, m.h_horizons, nadmit * sizeof(int32_t), cudaMemcpyHostToDevice, st));
      GROM_CUDA_TRY(
          cudaMemcpyAsync(m.d_u0, m.h_u0, (size_t)nadmit * m.n * sizeof(double), cudaMemcpyHostToDevice, st));
      GROM_CUDA_TRY(slot_admit_launch(m.traj->hist, m.traj->taken, m.traj->steps_left, m.traj->active, m.n, nadmit,
                                      m.d_slots, m.d_horizons, m.d_u0, st));
    }
    peak_bytes = std::max(peak_bytes, used);
    peak_active = std::max(peak_active, active_total);
    return GROM_OK;
  };

  while (finished < count) {
    const double t = now();
    while (next < order.size() && reqs[order[next]].arrival <= t) {
      const int q = order[next++];
      s->models[reqs[q].model].ready.push_back(q);
    }
    bool progressed = false;
    for (auto& m : s->models) {
      if (m.in_flight) {
        if (s->simulate) {
          if (vclock < m.sim_done) continue;
        } else {
          const cudaError_t qe = cudaEventQuery(m.done_ev);
          if (qe == cudaErrorNotReady) continue;
          if (qe != cudaSuccess) return cuda_fail(qe, "grom_serve");
        }
        m.in_flight = false;
        grom_status st = retire(m);
        if (st) return st;
        progressed = true;
      }
      grom_status st = admit(m, now());
      if (st) return st;
      bool any = false;
      for (int b = 0; b < m.slots && !any; ++b) any = m.slot_req[b] >= 0;
      if (!any) continue;
      ++quanta;
      progressed = true;
      m.in_flight = true;
      if (s->simulate) {
        m.sim_done = vclock + s->quantum * m.step_seconds;
        for (int b = 0; b < m.slots; ++b)
          if (m.slot_req[b] >= 0) m.sim_left[b] = std::max(0, m.sim_left[b] - s->quantum);
      } else {
        st = grom_step(m.traj, s->quantum, nullptr, nullptr);
        if (st) return st;
        cudaStream_t sm = m.rom->stream;
        GROM_CUDA_TRY(
            cudaMemcpyAsync(m.h_left, m.traj->steps_left, m.slots * sizeof(int32_t), cudaMemcpyDeviceToHost, sm));
        GROM_CUDA_TRY(
            cudaMemcpyAsync(m.h_taken, m.traj->taken, m.slots * sizeof(int64_t), cudaMemcpyDeviceToHost, sm));
        GROM_CUDA_TRY(cudaEventRecord(m.done_ev, sm));
      }
    }
    if (progressed || finished >= count) continue;
    // nothing could run: wait for the next event
    double t_next = next < order.size() ? reqs[order[next]].arrival : 1e300;
    bool busy = false;
    for (auto& m : s->models)
      if (m.in_flight) {
        busy = true;
        if (s->simulate) t_next = std::min(t_next, m.sim_done);
      }
    if (s->simulate) {
      if (t_next >= 1e299) return fail(GROM_ERR_INVALID_ARG, "grom_serve: no progress possible");
      vclock = std::max(vclock, t_next);
    } else if (!busy) {
      const double wait = t_next - now();
      if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(std::min(wait, 0.0005)));
    }
  }
  if (stats) {
    stats->trajectory_steps = tsteps;
    stats->quanta = quanta;
    stats->seconds = now();
    stats->peak_bytes = peak_bytes;
    stats->peak_active = peak_active;
    stats->reserved = 0;
  }
  return GROM_OK;
}

}  // extern "C"
