// Software-managed device cache of host fields (grid_dwf_cache_*; declared in include/grid_dwf.h).
//
// The paper (Section 2.3, "Memory models and software managed cache") keeps lattice data in host
// memory and moves whole fields to the accelerator when a view with an access intent is opened,
// with a device footprint capped by a high watermark and a least-recently-used replacement that
// it controls. This is that cache for the library's fields, for workloads whose fields do not all
// fit in HBM at once (many right-hand sides or pseudofermions, lattices larger than one GPU):
//   - an entry per host buffer: device buffer (or none), size, open-view count, priority, state:
//       EMPTY      no device copy (the host copy is the data),
//       CONSISTENT host and device copies equal,
//       CPU_DIRTY  the host copy is newer (the device copy is stale),
//       ACC_DIRTY  the device copy is newer (the host copy is stale);
//   - opening a view moves data as its intent needs (accelerator intents copy in a stale or
//     missing device copy, except write-discard; CPU intents copy back a newer device copy) and
//     moves the entry to the front of its LRU list; closing decrements the view count;
//   - before a device buffer is allocated, entries are evicted from the back of the LRU lists
//     (fields advised as infrequently used first) until the new buffer fits under the watermark;
//     an evicted ACC_DIRTY entry is copied back to the host first; entries with open views are
//     never evicted, and if nothing can be evicted the open fails with GRID_DWF_ERR_OOM.
// The data motion goes through a backend (device allocation, free and the two copies): CUDA by
// default (cudaMalloc, cudaFree, cudaMemcpyAsync on the cache's stream; the CPU intents wait for
// the stream), or caller-supplied functions, which lets the host logic run without a GPU.
#include <cuda_runtime.h>

#include <list>
#include <string>
#include <unordered_map>

#include "../../include/grid_dwf.h"

namespace {

enum State : int { EMPTY = 0, CONSISTENT = 1, CPU_DIRTY = 2, ACC_DIRTY = 3 };

struct Entry {
  void* host = nullptr;
  size_t bytes = 0;
  void* dev = nullptr;
  int state = EMPTY;
  int views = 0;         // open accelerator views (pin the device copy)
  int advice = GRID_DWF_ADVISE_NORMAL;
  bool in_lru = false;
  std::list<void*>::iterator lru_it;
};

int cuda_alloc(void*, size_t bytes, void** dev) { return cudaMalloc(dev, bytes) == cudaSuccess ? 0 : -1; }
int cuda_free(void*, void* dev) { return cudaFree(dev) == cudaSuccess ? 0 : -1; }

}  // namespace

struct grid_dwf_cache {
  size_t watermark = 0;
  size_t resident = 0;  // bytes of device buffers held
  cudaStream_t stream = nullptr;
  grid_dwf_cache_backend be{};
  bool cuda = true;
  std::unordered_map<void*, Entry> table;
  std::list<void*> lru[2];  // [advice]: front = most recently used
  grid_dwf_cache_stats st{};
  std::string err;
};

namespace {

int cfail(grid_dwf_cache* c, int code, const std::string& m) {
  c->err = m;
  return code;
}

int to_device(grid_dwf_cache* c, Entry& e) {
  c->st.bytes_to_device += e.bytes;
  ++c->st.copies_to_device;
  if (c->cuda)
    return cudaMemcpyAsync(e.dev, e.host, e.bytes, cudaMemcpyHostToDevice, c->stream) == cudaSuccess ? 0 : -1;
  return c->be.to_device(c->be.ctx, e.dev, e.host, e.bytes);
}

int to_host(grid_dwf_cache* c, Entry& e) {
  c->st.bytes_to_host += e.bytes;
  ++c->st.copies_to_host;
  if (c->cuda) {
    if (cudaMemcpyAsync(e.host, e.dev, e.bytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess) return -1;
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? 0 : -1;
  }
  return c->be.to_host(c->be.ctx, e.host, e.dev, e.bytes);
}

void touch(grid_dwf_cache* c, Entry& e) {
  auto& l = c->lru[e.advice];
  if (e.in_lru) l.erase(e.lru_it);
  l.push_front(e.host);
  e.lru_it = l.begin();
  e.in_lru = true;
}

// Release the device copy of an unpinned entry, writing it back first if it is the newer copy.
int evict(grid_dwf_cache* c, Entry& e) {
  if (e.state == ACC_DIRTY && to_host(c, e) != 0) return cfail(c, GRID_DWF_ERR_CUDA, "cache: copy back on eviction failed");
  if (c->cuda ? cuda_free(nullptr, e.dev) != 0 : c->be.free(c->be.ctx, e.dev) != 0)
    return cfail(c, GRID_DWF_ERR_CUDA, "cache: device free failed");
  c->resident -= e.bytes;
  e.dev = nullptr;
  e.state = EMPTY;
  ++c->st.evictions;
  return GRID_DWF_OK;
}

// Make room for `bytes` under the watermark: least recently used unpinned entries go first, the
// infrequently used list before the normal one.
int make_room(grid_dwf_cache* c, size_t bytes, const void* keep) {
  for (int pass = GRID_DWF_ADVISE_INFREQUENT; pass >= GRID_DWF_ADVISE_NORMAL && c->resident + bytes > c->watermark;
       --pass) {
    auto& l = c->lru[pass];  // holds exactly the entries with a device copy
    for (auto it = l.end(); it != l.begin() && c->resident + bytes > c->watermark;) {
      --it;
      Entry& v = c->table.at(*it);
      if (v.views > 0 || v.host == keep) continue;
      const int rc = evict(c, v);
      if (rc != GRID_DWF_OK) return rc;
      it = l.erase(it);  // the element after the erased one; the next step moves before it
      v.in_lru = false;
    }
  }
  if (c->resident + bytes > c->watermark)
    return cfail(c, GRID_DWF_ERR_OOM, "cache: the open views pin more than the watermark allows");
  return GRID_DWF_OK;
}

}  // namespace

extern "C" {

int grid_dwf_cache_create(size_t high_watermark, void* stream, const grid_dwf_cache_backend* backend,
                          grid_dwf_cache_t** out) {
  if (!out) return GRID_DWF_ERR_INVALID_ARG;
  *out = nullptr;
  if (high_watermark == 0) return GRID_DWF_ERR_INVALID_ARG;
  if (backend && (!backend->alloc || !backend->free || !backend->to_device || !backend->to_host))
    return GRID_DWF_ERR_INVALID_ARG;
  grid_dwf_cache* c = new grid_dwf_cache();
  c->watermark = high_watermark;
  c->stream = static_cast<cudaStream_t>(stream);
  if (backend) {
    c->be = *backend;
    c->cuda = false;
  }
  *out = c;
  return GRID_DWF_OK;
}

int grid_dwf_cache_destroy(grid_dwf_cache_t* c) {
  if (!c) return GRID_DWF_ERR_INVALID_ARG;
  if (c->cuda) cudaStreamSynchronize(c->stream);
  for (auto& kv : c->table)
    if (kv.second.dev) {
      if (c->cuda)
        cuda_free(nullptr, kv.second.dev);
      else
        c->be.free(c->be.ctx, kv.second.dev);
    }
  delete c;
  return GRID_DWF_OK;
}

int grid_dwf_cache_advise(grid_dwf_cache_t* c, void* host, size_t bytes, int advice) {
  if (!c || !host || bytes == 0) return GRID_DWF_ERR_INVALID_ARG;
  if (advice != GRID_DWF_ADVISE_NORMAL && advice != GRID_DWF_ADVISE_INFREQUENT)
    return cfail(c, GRID_DWF_ERR_INVALID_ARG, "cache: unknown advice");
  auto it = c->table.find(host);
  if (it == c->table.end()) {
    Entry e;
    e.host = host;
    e.bytes = bytes;
    e.advice = advice;
    c->table.emplace(host, e);
    return GRID_DWF_OK;
  }
  Entry& e = it->second;
  if (e.bytes != bytes) return cfail(c, GRID_DWF_ERR_INVALID_ARG, "cache: size differs from the registered field");
  if (e.in_lru && e.advice != advice) {
    c->lru[e.advice].erase(e.lru_it);
    e.in_lru = false;
    e.advice = advice;
    touch(c, e);
  }
  e.advice = advice;
  return GRID_DWF_OK;
}

int grid_dwf_cache_open(grid_dwf_cache_t* c, void* host, size_t bytes, int intent, void** ptr) {
  if (!c || !host || !ptr || bytes == 0) return GRID_DWF_ERR_INVALID_ARG;
  *ptr = nullptr;
  if (intent < GRID_DWF_CPU_READ || intent > GRID_DWF_ACC_WRITE_DISCARD)
    return cfail(c, GRID_DWF_ERR_INVALID_ARG, "cache: unknown intent");
  auto it = c->table.find(host);
  if (it == c->table.end()) {
    Entry e;
    e.host = host;
    e.bytes = bytes;
    it = c->table.emplace(host, e).first;
  }
  Entry& e = it->second;
  if (e.bytes != bytes) return cfail(c, GRID_DWF_ERR_INVALID_ARG, "cache: size differs from the registered field");
  if (intent == GRID_DWF_CPU_READ || intent == GRID_DWF_CPU_WRITE) {
    if (e.views > 0) return cfail(c, GRID_DWF_ERR_ALIAS, "cache: a CPU view while accelerator views are open");
    if (e.state == ACC_DIRTY) {
      if (to_host(c, e) != 0) return cfail(c, GRID_DWF_ERR_CUDA, "cache: copy to host failed");
      e.state = CONSISTENT;
    }
    if (intent == GRID_DWF_CPU_WRITE && e.dev) e.state = CPU_DIRTY;
    ++c->st.cpu_opens;
    *ptr = host;
    return GRID_DWF_OK;
  }
  // accelerator intents
  if (!e.dev) {
    ++c->st.misses;
    const int rc = make_room(c, e.bytes, host);
    if (rc != GRID_DWF_OK) return rc;
    const int arc = c->cuda ? cuda_alloc(nullptr, e.bytes, &e.dev) : c->be.alloc(c->be.ctx, e.bytes, &e.dev);
    if (arc != 0 || !e.dev) {
      e.dev = nullptr;
      return cfail(c, GRID_DWF_ERR_OOM, "cache: device allocation failed");
    }
    c->resident += e.bytes;
    if (c->resident > c->st.peak_resident) c->st.peak_resident = c->resident;
    e.state = CPU_DIRTY;  // a fresh buffer holds nothing yet
  } else {
    ++c->st.hits;
  }
  if (e.state == CPU_DIRTY && intent != GRID_DWF_ACC_WRITE_DISCARD) {
    if (to_device(c, e) != 0) return cfail(c, GRID_DWF_ERR_CUDA, "cache: copy to device failed");
    e.state = CONSISTENT;
  }
  if (intent != GRID_DWF_ACC_READ) e.state = ACC_DIRTY;
  ++e.views;
  touch(c, e);
  *ptr = e.dev;
  return GRID_DWF_OK;
}

int grid_dwf_cache_close(grid_dwf_cache_t* c, void* host) {
  if (!c || !host) return GRID_DWF_ERR_INVALID_ARG;
  auto it = c->table.find(host);
  if (it == c->table.end()) return cfail(c, GRID_DWF_ERR_INVALID_ARG, "cache: unknown field");
  if (it->second.views > 0) --it->second.views;
  return GRID_DWF_OK;
}

int grid_dwf_cache_flush(grid_dwf_cache_t* c) {
  if (!c) return GRID_DWF_ERR_INVALID_ARG;
  for (auto& kv : c->table) {
    Entry& e = kv.second;
    if (e.state == ACC_DIRTY && e.views == 0) {
      if (to_host(c, e) != 0) return cfail(c, GRID_DWF_ERR_CUDA, "cache: copy to host failed");
      e.state = CONSISTENT;
    }
  }
  return GRID_DWF_OK;
}

int grid_dwf_cache_forget(grid_dwf_cache_t* c, void* host) {
  if (!c || !host) return GRID_DWF_ERR_INVALID_ARG;
  auto it = c->table.find(host);
  if (it == c->table.end()) return GRID_DWF_OK;
  Entry& e = it->second;
  if (e.views > 0) return cfail(c, GRID_DWF_ERR_ALIAS, "cache: the field has open views");
  if (e.dev) {
    const int rc = evict(c, e);  // writes a newer device copy back first
    if (rc != GRID_DWF_OK) return rc;
    --c->st.evictions;  // not a replacement
  }
  if (e.in_lru) c->lru[e.advice].erase(e.lru_it);
  c->table.erase(it);
  return GRID_DWF_OK;
}

int grid_dwf_cache_query(const grid_dwf_cache_t* c, const void* host, int* state, int* views, void** dev) {
  if (!c || !host) return GRID_DWF_ERR_INVALID_ARG;
  auto it = c->table.find(const_cast<void*>(host));
  if (it == c->table.end()) return GRID_DWF_ERR_INVALID_ARG;
  if (state) *state = it->second.state;
  if (views) *views = it->second.views;
  if (dev) *dev = it->second.dev;
  return GRID_DWF_OK;
}

int grid_dwf_cache_get_stats(const grid_dwf_cache_t* c, grid_dwf_cache_stats* st) {
  if (!c || !st) return GRID_DWF_ERR_INVALID_ARG;
  *st = c->st;
  st->resident_bytes = c->resident;
  return GRID_DWF_OK;
}

const char* grid_dwf_cache_last_error(const grid_dwf_cache_t* c) { return c ? c->err.c_str() : "null cache"; }

}  // extern "C"
