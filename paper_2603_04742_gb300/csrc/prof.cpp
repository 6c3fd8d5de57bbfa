// Per-kernel device timing with CUDA events (see Profiler in internal.h).
#include "internal.h"

namespace hespmv {

int prof_begin(const Ctx &c, const char *name, cudaStream_t st) {
    Profiler *p = c.c->prof;
    if (!p || !p->on) return -1;
    auto it = p->ids.find(name);
    int kind;
    if (it == p->ids.end()) {
        kind = (int)p->names.size();
        p->ids[name] = kind;
        p->names.push_back(name);
    } else {
        kind = it->second;
    }
    while (p->pool.size() < p->used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        p->pool.push_back(e);
    }
    Profiler::Rec r{kind, p->pool[p->used], p->pool[p->used + 1]};
    p->used += 2;
    cudaEventRecord(r.a, st);
    p->recs.push_back(r);
    return (int)p->recs.size() - 1;
}

void prof_end(const Ctx &c, int rec, cudaStream_t st) {
    Profiler *p = c.c->prof;
    if (!p || rec < 0 || rec >= (int)p->recs.size()) return;
    cudaEventRecord(p->recs[rec].b, st);
}

cudaError_t Profiler::collect() {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    launches.resize(names.size(), 0);
    ms.resize(names.size(), 0.0);
    for (const Rec &r : recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            launches[r.kind] += 1;
            ms[r.kind] += t;
        }
    }
    recs.clear();
    used = 0;
    return cudaSuccess;
}

void Profiler::reset() {
    recs.clear();
    used = 0;
    names.clear();
    ids.clear();
    launches.clear();
    ms.clear();
}

Profiler::~Profiler() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace hespmv
