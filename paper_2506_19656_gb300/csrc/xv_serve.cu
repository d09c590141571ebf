// xv_serve.cu -- serving: a request loop with continuous batching.
//
// Requests carry a cube in HOST memory.  A library thread admits them in
// arrival order while a slot is free and their device buffers fit the
// context's memory budget; admission uploads the cube and quantises it on a
// copy stream, so it overlaps whatever is running.  The loop then runs ticks:
// one persistent launch advances every ready request by up to
// `frames_per_tick` frames (its frames [t, t + k) go through the same
// data-flow kernel as xv_encode_batch, frame t - 1 being complete from the
// previous tick).  Requests join and leave between ticks -- continuous
// batching at frame granularity -- and keep their planes and reference frames
// resident in the meantime.  A request that reaches its last frame gets its
// PSNR and rate read back, its reconstruction and vectors copied out if asked
// for, and its device memory released; the result records the latency from
// submission to completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "me.cuh"
#include "tqr.cuh"
#include "xv_internal.h"

namespace xvh {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

enum class RState { Pending, Loading, Active, Done };

struct Request {
    uint64_t ticket = 0;
    xv_request r{};
    RState state = RState::Pending;
    bool cancel = false;
    double t_arrival = 0.0;
    xv_result res{};
    // device buffers (one allocation)
    unsigned char* dbuf = nullptr;
    size_t dbytes = 0;
    void* d_src = nullptr;
    uint16_t *d_planes = nullptr, *d_recon = nullptr;
    int16_t* d_mv = nullptr;
    uint64_t* d_bits = nullptr;
    double* d_minmax = nullptr;
    unsigned* d_enc = nullptr;
    BandQ* d_bq = nullptr;
    unsigned *d_rows = nullptr, *d_deps = nullptr;
    PsnrPart *d_part = nullptr, *d_out = nullptr;
    int G = 0, Hp = 0, Wp = 0, nx = 0, ny = 0, nblk = 0;
    int t_next = 0;
    cudaEvent_t ready = nullptr;
    std::string err;  // the message of a failed request (from the serving thread)
};

size_t request_bytes(const xv_request& q, int* G_, int* Hp_, int* Wp_, int* nblk_) {
    const int ctu = q.p.ctu, G = (q.bands + 2) / 3;
    const int Hp = (q.H + ctu - 1) / ctu * ctu, Wp = (q.W + ctu - 1) / ctu * ctu;
    const int64_t npu = (int64_t)(Hp / ctu) * (Wp / ctu), fr = (int64_t)G * q.T;
    const int nblk = psnr_blocks_per_band((int64_t)q.T * q.H * q.W, q.bands);
    const size_t esz = q.dtype == XV_F32 ? 4 : 2;
    size_t b = 0;
    b += align256(esz * (size_t)q.bands * q.T * q.H * q.W);    // source
    b += 2 * align256((size_t)fr * 3 * Hp * Wp * 2);            // planes, recon
    b += align256((size_t)fr * npu * 4);                        // motion vectors
    b += align256((size_t)fr * 8);                              // bits
    b += align256((size_t)q.bands * 16) + align256((size_t)q.bands * 8) + align256(sizeof(BandQ) * q.bands);
    b += 2 * align256((size_t)fr * (Hp / ctu) * 4);             // row and dependency counters
    b += align256(sizeof(PsnrPart) * (size_t)q.bands * nblk) + align256(sizeof(PsnrPart) * q.bands);
    if (G_) *G_ = G;
    if (Hp_) *Hp_ = Hp;
    if (Wp_) *Wp_ = Wp;
    if (nblk_) *nblk_ = nblk;
    return b;
}

}  // namespace

struct ServeState {
    int device = 0;
    int max_slots = 0, frames_per_tick = 0;
    size_t budget = 0, in_use = 0;
    long long wait_budget = 0;
    int block[4] = {256, 256, 256, 256};  // persistent block size per CTU class (8, 16, 32, 64)
    int per_cap[4] = {0, 0, 0, 0};        // resident-block cap per SM (0: as many as fit)
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    bool stop = false;
    std::deque<Request*> pending;
    std::vector<Request*> active;              // admitted, not finished
    std::map<uint64_t, Request*> by_ticket;
    uint64_t next_ticket = 1;
    cudaStream_t s_copy = nullptr, s_tick = nullptr;
    // tick scratch
    JobDev* d_jobs = nullptr;
    ClassDev* d_cls = nullptr;
    BatchCtl* d_ctl = nullptr;
    uint64_t* d_queue = nullptr;
    size_t queue_cap = 0;
    unsigned long long* d_totals = nullptr;
    JobDev* h_jobs = nullptr;                  // pinned
    unsigned char* h_res = nullptr;            // pinned: ctl, totals, per-slot PSNR/bands
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    uint64_t ticks = 0;
    double kernel_ms = 0.0;
    int peak_active = 0;
    xv_status fatal = XV_OK;

    void loop();
    bool admit_locked();
    void finish(Request* q, xv_status st);
};

static constexpr size_t kResSlotBytes = (sizeof(PsnrPart) + sizeof(BandQ)) * XV_MAX_BANDS;

void ServeState::finish(Request* q, xv_status st) {
    // caller holds the lock
    q->res.status = st;
    q->res.latency_s = now_s() - q->t_arrival;
    if (st != XV_OK) q->err = last_error_text();
    q->state = RState::Done;
    if (q->dbuf) {
        cudaFreeAsync(q->dbuf, s_tick);
        in_use -= q->dbytes;
        q->dbuf = nullptr;
    }
    if (q->ready) { cudaEventDestroy(q->ready); q->ready = nullptr; }
}

// Admit pending requests while a slot and the memory budget allow (lock held).
bool ServeState::admit_locked() {
    bool any = false;
    while (!pending.empty() && (int)active.size() < max_slots) {
        Request* q = pending.front();
        if (q->cancel) {
            pending.pop_front();
            finish(q, XV_ECANCELLED);
            continue;
        }
        int G, Hp, Wp, nblk;
        const size_t need = request_bytes(q->r, &G, &Hp, &Wp, &nblk);
        if (budget && need > budget) {
            pending.pop_front();
            set_error("request needs %zu bytes, more than the whole budget", need);
            finish(q, XV_EBUDGET);
            continue;
        }
        if (budget && in_use + need > budget) break;  // wait until memory frees up
        void* mem = nullptr;
        if (cudaMallocAsync(&mem, need, s_copy) != cudaSuccess) {
            cudaGetLastError();
            if (active.empty()) {
                pending.pop_front();
                finish(q, XV_ENOMEM);
                continue;
            }
            break;
        }
        pending.pop_front();
        in_use += need;
        q->dbuf = (unsigned char*)mem;
        q->dbytes = need;
        q->G = G; q->Hp = Hp; q->Wp = Wp; q->nblk = nblk;
        q->nx = Wp / q->r.p.ctu;
        q->ny = Hp / q->r.p.ctu;
        const xv_request& r = q->r;
        const int64_t npu = (int64_t)q->nx * q->ny, fr = (int64_t)G * r.T;
        const size_t esz = r.dtype == XV_F32 ? 4 : 2;
        unsigned char* p = q->dbuf;
        auto take = [&](size_t b) { unsigned char* o = p; p += align256(b); return o; };
        q->d_src = take(esz * (size_t)r.bands * r.T * r.H * r.W);
        q->d_planes = (uint16_t*)take((size_t)fr * 3 * Hp * Wp * 2);
        q->d_recon = (uint16_t*)take((size_t)fr * 3 * Hp * Wp * 2);
        q->d_mv = (int16_t*)take((size_t)fr * npu * 4);
        q->d_bits = (uint64_t*)take((size_t)fr * 8);
        q->d_minmax = (double*)take((size_t)r.bands * 16);
        q->d_enc = (unsigned*)take((size_t)r.bands * 8);
        q->d_bq = (BandQ*)take(sizeof(BandQ) * r.bands);
        q->d_rows = (unsigned*)take((size_t)fr * q->ny * 4);
        q->d_deps = (unsigned*)take((size_t)fr * q->ny * 4);
        q->d_part = (PsnrPart*)take(sizeof(PsnrPart) * (size_t)r.bands * nblk);
        q->d_out = (PsnrPart*)take(sizeof(PsnrPart) * r.bands);
        cudaError_t e = cudaMemcpyAsync(q->d_src, r.src, esz * (size_t)r.bands * r.T * r.H * r.W,
                                        cudaMemcpyHostToDevice, s_copy);
        if (e == cudaSuccess)
            e = launch_prepare_bands(q->d_src, r.dtype, r.bands, (int64_t)r.T * r.H * r.W, q->d_minmax, 0, q->d_enc,
                                     q->d_bq, s_copy);
        if (e == cudaSuccess)
            e = launch_quantize_pack(q->d_src, r.dtype, r.bands, r.T, r.H, r.W, Hp, Wp, q->d_bq, q->d_planes, s_copy);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(q->ready, s_copy);
        if (e != cudaSuccess) {
            cudaGetLastError();
            set_error("request upload: %s", cudaGetErrorString(e));
            finish(q, XV_ECUDA);
            continue;
        }
        q->state = RState::Loading;
        active.push_back(q);
        any = true;
    }
    peak_active = std::max(peak_active, (int)active.size());
    return any;
}

void ServeState::loop() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<Request*> tick;
        {
            std::unique_lock<std::mutex> lk(mu);
            admit_locked();
            // drop cancelled requests at the tick boundary
            for (size_t i = 0; i < active.size();) {
                if (active[i]->cancel) {
                    // its upload may still be in flight on the copy stream
                    if (active[i]->ready) cudaEventSynchronize(active[i]->ready);
                    finish(active[i], XV_ECANCELLED);
                    active.erase(active.begin() + i);
                } else {
                    ++i;
                }
            }
            for (Request* q : active) {
                if (q->state == RState::Loading && cudaEventQuery(q->ready) == cudaSuccess) q->state = RState::Active;
                if (q->state == RState::Active) tick.push_back(q);
            }
            if (tick.empty()) {
                if (stop && active.empty()) break;
                cv.wait_for(lk, std::chrono::microseconds(active.empty() ? 2000 : 50));
                continue;
            }
        }
        // ---- one tick over the ready requests (outside the lock)
        const int n = (int)tick.size();
        size_t total[4] = {0, 0, 0, 0}, nfirst[4] = {0, 0, 0, 0}, smem[4] = {0, 0, 0, 0};
        for (int i = 0; i < n; ++i) {
            Request* q = tick[i];
            const xv_request& r = q->r;
            const int k = r.p.ctu == 8 ? 0 : r.p.ctu == 16 ? 1 : r.p.ctu == 32 ? 2 : 3;
            const int tb = q->t_next, te = std::min(r.T, tb + frames_per_tick);
            const int64_t npu = (int64_t)q->nx * q->ny;
            total[k] += (size_t)q->G * (te - tb) * npu;
            nfirst[k] += (size_t)q->G * npu;
            smem[k] = std::max(smem[k], persist_smem_bytes(r.p.ctu, r.p.search_range, true));
        }
        ClassDev cls[4];
        size_t tot = 0;
        for (int k = 0; k < 4; ++k) {
            cls[k] = ClassDev{(int64_t)tot, (unsigned)total[k], (unsigned)nfirst[k]};
            tot += total[k];
        }
        cudaError_t e = cudaSuccess;
        if (tot > queue_cap) {
            if (d_queue) cudaFreeAsync(d_queue, s_tick);
            d_queue = nullptr;
            queue_cap = 0;
            e = cudaMallocAsync(&d_queue, sizeof(uint64_t) * tot * 2, s_tick);
            if (e == cudaSuccess) queue_cap = tot * 2;
        }
        size_t qnext[4];
        for (int k = 0; k < 4; ++k) qnext[k] = (size_t)cls[k].qoff;
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            Request* q = tick[i];
            const xv_request& r = q->r;
            const int k = r.p.ctu == 8 ? 0 : r.p.ctu == 16 ? 1 : r.p.ctu == 32 ? 2 : 3;
            // h_jobs is raw pinned memory: start every record from its
            // defaults, then fill it
            JobDev& d = h_jobs[i];
            d = JobDev{};
            d.planes = q->d_planes;
            d.recon = q->d_recon;
            d.mv = q->d_mv;
            d.cost = nullptr;
            d.levels = nullptr;
            d.tu = nullptr;
            d.bits = q->d_bits;
            d.rowdone = q->d_rows;
            d.depcnt = q->d_deps;
            d.lf8 = r.p.lambda_fp8;
            d.lmv = r.p.lambda_mv_fp16;
            d.G = q->G; d.T = r.T; d.Hp = q->Hp; d.Wp = q->Wp; d.ctu = r.p.ctu; d.R = r.p.search_range; d.qp = r.p.qp;
            d.tu_mask = r.p.tu_mask;
            d.nx = q->nx;
            d.ny = q->ny;
            d.qfirst = (int64_t)qnext[k];
            d.tb = q->t_next;
            d.te = std::min(r.T, q->t_next + frames_per_tick);
            qnext[k] += (size_t)q->G * q->nx * q->ny;
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_jobs, h_jobs, sizeof(JobDev) * n, cudaMemcpyHostToDevice, s_tick);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_cls, cls, sizeof cls, cudaMemcpyHostToDevice, s_tick);
        if (e == cudaSuccess) e = launch_batch_prologue(d_jobs, n, d_cls, d_queue, d_ctl, wait_budget, -1, s_tick);
        if (e == cudaSuccess) e = cudaEventRecord(ev0, s_tick);
        const int ctus[4] = {8, 16, 32, 64};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
            if (!total[k]) continue;
            const int grid = persist_grid(ctus[k], block[k], smem[k], false, per_cap[k]);
            e = launch_persist(ctus[k], block[k], false, d_jobs, d_queue + cls[k].qoff, d_ctl + k, smem[k], grid,
                               s_tick);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev1, s_tick);
        // results of the requests this tick finishes
        if (e == cudaSuccess) e = launch_bits_totals(d_jobs, n, d_totals, s_tick);
        BatchCtl* h_ctl = (BatchCtl*)h_res;
        unsigned long long* h_tot = (unsigned long long*)(h_res + sizeof(BatchCtl) * 4);
        unsigned char* h_slots = h_res + sizeof(BatchCtl) * 4 + sizeof(unsigned long long) * 256;
        for (int i = 0; i < n && e == cudaSuccess; ++i) {
            Request* q = tick[i];
            const xv_request& r = q->r;
            if (h_jobs[i].te != r.T) continue;
            e = launch_psnr(q->d_src, r.dtype, r.bands, r.T, r.H, r.W, q->d_planes, q->d_recon, q->Hp, q->Wp, q->d_bq,
                            q->d_part, q->nblk, q->d_out, s_tick);
            unsigned char* slot = h_slots + kResSlotBytes * i;
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot, q->d_out, sizeof(PsnrPart) * r.bands, cudaMemcpyDeviceToHost, s_tick);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(slot + sizeof(PsnrPart) * XV_MAX_BANDS, q->d_bq, sizeof(BandQ) * r.bands,
                                    cudaMemcpyDeviceToHost, s_tick);
            if (e == cudaSuccess && r.recon_out)
                e = cudaMemcpyAsync(r.recon_out, q->d_recon, (size_t)q->G * r.T * 3 * q->Hp * q->Wp * 2,
                                    cudaMemcpyDeviceToHost, s_tick);
            if (e == cudaSuccess && r.mv_out)
                e = cudaMemcpyAsync(r.mv_out, q->d_mv, (size_t)q->G * r.T * q->nx * q->ny * 4, cudaMemcpyDeviceToHost,
                                    s_tick);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_ctl, d_ctl, sizeof(BatchCtl) * 4, cudaMemcpyDeviceToHost, s_tick);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_tot, d_totals, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost, s_tick);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s_tick);
        float kms = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&kms, ev0, ev1) == cudaSuccess) kernel_ms += kms;
        std::lock_guard<std::mutex> lk(mu);
        ++ticks;
        int err = 0;
        for (int k = 0; k < 4; ++k)
            if (e == cudaSuccess && total[k] && h_ctl[k].err) err = h_ctl[k].err;
        if (e != cudaSuccess || err) {
            if (e != cudaSuccess) {
                cudaGetLastError();
                set_error("serving tick: %s", cudaGetErrorString(e));
            } else {
                set_error("serving tick: device status %d", err);
            }
            const xv_status st = e != cudaSuccess ? XV_ECUDA : (xv_status)err;
            for (Request* q : tick) {
                finish(q, st);
                active.erase(std::find(active.begin(), active.end(), q));
            }
            if (e != cudaSuccess) { fatal = st; stop = true; }
            cv.notify_all();
            continue;
        }
        for (int i = 0; i < n; ++i) {
            Request* q = tick[i];
            const xv_request& r = q->r;
            q->t_next = h_jobs[i].te;
            if (q->t_next != r.T) continue;
            const PsnrPart* o = (const PsnrPart*)(h_slots + kResSlotBytes * i);
            const BandQ* bq = (const BandQ*)(h_slots + kResSlotBytes * i + sizeof(PsnrPart) * XV_MAX_BANDS);
            double acc = 0.0;
            bool inf = false;
            for (int b = 0; b < r.bands; ++b) {
                const double cnt = (double)o[b].count;
                const double m = cnt > 0 ? o[b].sse / cnt : 0.0;
                const double peak = bq[b].hi > 0.0 ? bq[b].hi : bq[b].hi - bq[b].lo;
                const double p = m > 0.0 ? 10.0 * std::log10(peak * peak / m) : INFINITY;
                q->res.psnr_band[b] = p;
                q->res.mse_band[b] = m;
                q->res.sse10_band[b] = o[b].sse10;
                if (std::isinf(p)) inf = true; else acc += p;
            }
            q->res.psnr_mean = inf ? INFINITY : acc / r.bands;
            q->res.total_bits = h_tot[i];
            q->res.bands = r.bands;
            q->res.bpppb = (double)h_tot[i] / ((double)r.H * r.W * r.T * r.bands);
            q->res.ctu = r.p.ctu;
            q->res.block_size = block[r.p.ctu == 8 ? 0 : r.p.ctu == 16 ? 1 : r.p.ctu == 32 ? 2 : 3];
            finish(q, XV_OK);
            active.erase(std::find(active.begin(), active.end(), q));
        }
        cv.notify_all();
    }
}

ServeState* serve_create(int device, int max_slots, int frames_per_tick, size_t budget, long long wait_budget,
                         const int block[4], const int per_cap[4], xv_status* st) {
    ServeState* s = new ServeState;
    for (int k = 0; k < 4; ++k) {
        s->block[k] = block[k];
        s->per_cap[k] = per_cap[k];
    }
    s->device = device;
    s->max_slots = max_slots;
    s->frames_per_tick = frames_per_tick;
    s->budget = budget;
    s->wait_budget = wait_budget;
    cudaError_t e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_tick, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_jobs, sizeof(JobDev) * 256);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_cls, sizeof(ClassDev) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_ctl, sizeof(BatchCtl) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_totals, sizeof(unsigned long long) * 256);
    if (e == cudaSuccess) e = cudaMallocHost(&s->h_jobs, sizeof(JobDev) * 256);
    if (e == cudaSuccess)
        e = cudaMallocHost(&s->h_res, sizeof(BatchCtl) * 4 + sizeof(unsigned long long) * 256 + kResSlotBytes * 256);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&s->ev1);
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "serving set-up");
        return s;
    }
    *st = XV_OK;
    s->th = std::thread([s] { s->loop(); });
    return s;
}

void serve_destroy(ServeState* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Request* q : s->pending) q->cancel = true;
        for (Request* q : s->active) q->cancel = true;
    }
    s->cv.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->device);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (Request* q : s->pending) s->finish(q, XV_ECANCELLED);
        s->pending.clear();
    }
    if (s->s_tick) cudaStreamSynchronize(s->s_tick);
    if (s->s_copy) cudaStreamSynchronize(s->s_copy);
    for (auto& kv : s->by_ticket) delete kv.second;
    if (s->d_queue) cudaFree(s->d_queue);
    cudaFree(s->d_jobs);
    cudaFree(s->d_cls);
    cudaFree(s->d_ctl);
    cudaFree(s->d_totals);
    cudaFreeHost(s->h_jobs);
    cudaFreeHost(s->h_res);
    if (s->ev0) cudaEventDestroy(s->ev0);
    if (s->ev1) cudaEventDestroy(s->ev1);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    if (s->s_tick) cudaStreamDestroy(s->s_tick);
    delete s;
}

xv_status serve_submit(ServeState* s, const xv_request* r, uint64_t* ticket) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal) { set_error("serving stopped after an error"); return s->fatal; }
    if (s->stop) { set_error("serving is stopping"); return XV_EINVAL; }
    if (s->pending.size() >= 65536) { set_error("serving queue full"); return XV_EBUSY; }
    Request* q = new Request;
    q->ticket = s->next_ticket++;
    q->r = *r;
    q->t_arrival = now_s();
    s->pending.push_back(q);
    s->by_ticket[q->ticket] = q;
    *ticket = q->ticket;
    s->cv.notify_all();
    return XV_OK;
}

xv_status serve_poll(ServeState* s, uint64_t ticket, xv_result* res, int* done) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return XV_ENOTFOUND; }
    Request* q = it->second;
    *done = q->state == RState::Done;
    if (*done) {
        if (res) *res = q->res;
        if (q->res.status != XV_OK) set_error("%s", q->err.c_str());  // for the polling thread
        s->by_ticket.erase(it);
        delete q;
    }
    return XV_OK;
}

xv_status serve_cancel(ServeState* s, uint64_t ticket) {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return XV_ENOTFOUND; }
    it->second->cancel = true;
    s->cv.notify_all();
    return XV_OK;
}

void serve_stats(ServeState* s, uint64_t* ticks, double* kernel_ms, int* peak_active, size_t* bytes_in_use) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticks) *ticks = s->ticks;
    if (kernel_ms) *kernel_ms = s->kernel_ms;
    if (peak_active) *peak_active = s->peak_active;
    if (bytes_in_use) *bytes_in_use = s->in_use;
}

}  // namespace xvh
