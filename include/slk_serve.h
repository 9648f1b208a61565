/*
 * slk_serve.h -- request serving for the sliced kernel summation library.
 *
 * A server runs kernel-sum requests (the problem of Section 3: sources x with
 * weights w, targets y, a kernel and P slices) of uneven sizes concurrently on
 * one GPU.  Requests are admitted in arrival order while the device-memory
 * budget allows (each request reserves a conservative estimate of the memory
 * its plan and sum need, see slk_request_bytes), run on one of several worker
 * streams so that the kernels of different requests overlap on the device, and
 * release their reservation when they finish; a request that arrives while
 * others run starts as soon as a worker and memory are free.  Requests that
 * name the same nonzero source_key reuse one cached plan (the source side of
 * every slice is computed once), so repeated queries against the same x cost
 * only their target side; queued requests on the same cached plan are served
 * together by one sum over their concatenated targets (a request waiting for a
 * plan that another request is building stays queued without holding up the
 * requests behind it).
 *
 * Ownership: the caller owns x, w, y, s and the descriptor's directions array
 * and keeps them valid and unchanged until the request has been polled as
 * finished (a queued request reads them only when it starts).  Pointers may be host or
 * device pointers (as in slk.h).  A cached plan keeps no pointer to x or w.
 */
#ifndef SLK_SERVE_H
#define SLK_SERVE_H

#include "slk.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t workers;          /* concurrent requests (worker threads and streams); 0 = 4 */
    int64_t memory_budget;    /* device bytes requests may reserve; 0 = 80% of the free memory */
    int64_t plan_cache_bytes; /* device bytes cached plans may hold (within the budget); 0 = budget / 4 */
    int32_t reserved[8];
} slk_serve_desc;

typedef struct {
    slk_plan_desc desc;       /* kernel, parameter, P, precision, ... (as for slk_plan_create) */
    const void* x;            /* N x d sources (row stride ldx) */
    int64_t N, ldx;
    const void* w;            /* N weights */
    const void* y;            /* M x d targets (row stride ldy) */
    int64_t M, ldy;
    void* s;                  /* M outputs */
    uint64_t source_key;      /* nonzero: cache the plan under this key and reuse it for later
                                 requests with the same key (the caller guarantees the same x, w
                                 and descriptor); 0: no caching */
} slk_request;

typedef struct {
    slk_status status;        /* status of the request (SLK_OK, or the failing call's status) */
    int32_t plan_cached;      /* 1 if a cached plan served the request */
    int32_t batch_requests;   /* requests served by the same sum (the queued requests on one
                                 cached plan are batched: their targets are concatenated into
                                 one sum); 1 = alone */
    double queue_ms;          /* submission -> admission */
    double run_ms;            /* admission -> finished (plan, sum and synchronisation) */
    double total_ms;          /* submission -> finished */
    char message[128];        /* detail of a failure ("" when OK) */
} slk_result;

typedef struct slk_server_s* slk_server;

/* Create a server on the current device.  desc may be NULL (defaults). */
slk_status slk_serve_create(slk_server* server, const slk_serve_desc* desc);

/*
 * Queue a request; *id receives its identifier.  Returns SLK_ERR_INVALID for a
 * malformed request and SLK_ERR_OOM when its estimate exceeds the whole budget
 * (it could never be admitted); otherwise the request is queued.
 */
slk_status slk_serve_submit(slk_server server, const slk_request* request, uint64_t* id);

/*
 * Wait up to timeout_us microseconds (0: do not wait, < 0: wait without limit)
 * for request id.  SLK_OK with *result filled when it has finished (the
 * request is then forgotten), SLK_ERR_TIMEOUT when it is still queued or
 * running, SLK_ERR_NOT_FOUND for an unknown (or already polled) id.
 */
slk_status slk_serve_poll(slk_server server, uint64_t id, int64_t timeout_us, slk_result* result);

/* Conservative device bytes a request needs (plan build plus one sum); host-only. */
int64_t slk_request_bytes(const slk_plan_desc* desc, int64_t N, int64_t M);

/* Wait for all queued and running requests, then release the server and its cached plans. */
slk_status slk_serve_destroy(slk_server server);

#ifdef __cplusplus
}
#endif

#endif /* SLK_SERVE_H */
