// Online tile autotuner for batched launches.
//
// A tuned launch site has one launch parameter (an x chunk, a smoother form)
// whose candidate values tile the same work differently and compute bitwise
// the same result.  For each (site, n, B) the tuner hands out the candidates
// in turn on successive real launches, times each launch with a pair of CUDA
// events on the launching stream, reads the timings back once the events have
// completed (no host synchronisation: a pending pair is simply read at a later
// call), and after kSamples timings per candidate keeps the fastest (the
// minimum of its samples, which discards the first launch's one-time costs).
// While a stream is being captured into a CUDA graph nothing is timed or
// queried: the site gets the choice made so far, else its default.
#include <mutex>

#include "pm_internal.cuh"

namespace pmgb {

namespace {

constexpr int kMaxCand = 4, kSamples = 2, kSlots = 8, kEntries = 64;

struct Entry {
  int site = -1, n = 0, B = 0, dev = 0;   // key (events belong to device dev)
  int ncand = 0, cand[kMaxCand] = {};
  int chosen = -1;                    // index into cand once decided
  float best[kMaxCand] = {};          // minimum sample per candidate
  int count[kMaxCand] = {};           // samples read per candidate
  int slot_cand[kSlots] = {};         // candidate of a pending timing, -1 if free
  cudaEvent_t ev0[kSlots] = {}, ev1[kSlots] = {};
};

struct Ticket {
  int entry = -1, slot = -1;
};

std::mutex g_mu;
Entry g_tab[kEntries];
int g_used = 0;
int g_mode = 1;   // 0: defaults only, 1: tune batched launches
thread_local Ticket t_ticket;

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;   // unknown: behave as under capture (no events, no queries)
  }
  return st != cudaStreamCaptureStatusNone;
}

// Reads the completed timings of e; leaves pending ones for a later call.
// cudaEventQuery's "not ready" is not an error: it is cleared again, and only
// queried when no earlier error is waiting to be reported.
void harvest(Entry& e) {
  for (int k = 0; k < kSlots; ++k) {
    if (e.slot_cand[k] < 0) continue;
    if (cudaPeekAtLastError() != cudaSuccess) return;
    const cudaError_t q = cudaEventQuery(e.ev1[k]);
    if (q == cudaErrorNotReady) {
      cudaGetLastError();
      continue;
    }
    if (q != cudaSuccess) return;   // left for the library's own error check
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, e.ev0[k], e.ev1[k]) != cudaSuccess) {
      cudaGetLastError();
      e.slot_cand[k] = -1;
      continue;
    }
    const int c = e.slot_cand[k];
    e.best[c] = e.count[c] == 0 ? ms : fminf(e.best[c], ms);
    ++e.count[c];
    e.slot_cand[k] = -1;
  }
  bool done = true;
  for (int c = 0; c < e.ncand; ++c) done = done && e.count[c] >= kSamples;
  if (done) {
    int b = 0;
    for (int c = 1; c < e.ncand; ++c)
      if (e.best[c] < e.best[b]) b = c;
    e.chosen = b;
  }
}

Entry* find(int site, int n, int B, int dev, const int* cand, int ncand) {
  for (int i = 0; i < g_used; ++i)
    if (g_tab[i].site == site && g_tab[i].n == n && g_tab[i].B == B && g_tab[i].dev == dev) return &g_tab[i];
  if (g_used == kEntries) return nullptr;
  Entry& e = g_tab[g_used++];
  e.site = site;
  e.n = n;
  e.B = B;
  e.dev = dev;
  e.ncand = ncand;
  for (int c = 0; c < ncand; ++c) e.cand[c] = cand[c];
  for (int k = 0; k < kSlots; ++k) e.slot_cand[k] = -1;
  return &e;
}

}  // namespace

int tune_begin(int site, int n, int B, const int* cand, int ncand, int dflt, cudaStream_t s) {
  t_ticket = Ticket{};
  if (ncand <= 1 || ncand > kMaxCand) return ncand == 1 ? cand[0] : dflt;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_mode == 0) return dflt;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return dflt;
  }
  Entry* e = find(site, n, B, dev, cand, ncand);
  if (!e) return dflt;
  if (e->chosen >= 0) return e->cand[e->chosen];
  const bool cap = capturing(s);
  if (!cap) harvest(*e);
  if (e->chosen >= 0) return e->cand[e->chosen];
  if (cap) {   // best so far, else the default
    int b = -1;
    for (int c = 0; c < e->ncand; ++c)
      if (e->count[c] > 0 && (b < 0 || e->best[c] < e->best[b])) b = c;
    return b >= 0 ? e->cand[b] : dflt;
  }
  // the candidate with the fewest samples read or pending
  int pend[kMaxCand] = {};
  int slot = -1;
  for (int k = 0; k < kSlots; ++k) {
    if (e->slot_cand[k] >= 0) ++pend[e->slot_cand[k]];
    else if (slot < 0) slot = k;
  }
  int c = 0;
  for (int i = 1; i < e->ncand; ++i)
    if (e->count[i] + pend[i] < e->count[c] + pend[c]) c = i;
  if (slot < 0 || e->count[c] + pend[c] >= kSamples) return e->cand[c];   // all samples in flight
  if (!e->ev0[slot]) {
    if (cudaEventCreate(&e->ev0[slot]) != cudaSuccess || cudaEventCreate(&e->ev1[slot]) != cudaSuccess) {
      cudaGetLastError();
      return e->cand[c];
    }
  }
  if (cudaEventRecord(e->ev0[slot], s) != cudaSuccess) {
    cudaGetLastError();
    return e->cand[c];
  }
  e->slot_cand[slot] = c;
  t_ticket = Ticket{(int)(e - g_tab), slot};
  return e->cand[c];
}

bool tune_active() { return t_ticket.entry >= 0; }

void tune_end(cudaStream_t s) {
  const Ticket t = t_ticket;
  t_ticket = Ticket{};
  if (t.entry < 0) return;
  std::lock_guard<std::mutex> lock(g_mu);
  Entry& e = g_tab[t.entry];
  if (cudaEventRecord(e.ev1[t.slot], s) != cudaSuccess) {
    cudaGetLastError();
    e.slot_cand[t.slot] = -1;
  }
}

}  // namespace pmgb

using namespace pmgb;

extern "C" {

pm_status pm_autotune(int mode) {
  if (mode < 0 || mode > 2) return PM_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (mode == 2) {   // forget every choice and timing (events are kept for reuse)
    for (int i = 0; i < g_used; ++i) {
      Entry& e = g_tab[i];
      e.chosen = -1;
      for (int c = 0; c < kMaxCand; ++c) {
        e.best[c] = 0.0f;
        e.count[c] = 0;
      }
      for (int k = 0; k < kSlots; ++k) e.slot_cand[k] = -1;
    }
    g_mode = 1;
  } else {
    g_mode = mode;
  }
  return PM_OK;
}

int pm_autotune_report(int* out, int cap) {
  std::lock_guard<std::mutex> lock(g_mu);
  int dev = -1;
  if (g_used > 0 && cudaGetDevice(&dev) != cudaSuccess) cudaGetLastError();
  for (int i = 0; i < g_used; ++i)
    if (g_tab[i].dev == dev) harvest(g_tab[i]);
  const int m = g_used < cap ? g_used : cap;
  for (int i = 0; out && i < m; ++i) {
    const Entry& e = g_tab[i];
    int samples = 0;
    for (int c = 0; c < e.ncand; ++c) samples += e.count[c];
    out[5 * i + 0] = e.site;
    out[5 * i + 1] = e.n;
    out[5 * i + 2] = e.B;
    out[5 * i + 3] = e.chosen >= 0 ? e.cand[e.chosen] : -1;
    out[5 * i + 4] = samples;
  }
  return g_used;
}

}  // extern "C"
