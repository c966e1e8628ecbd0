/* lpb_serve.h -- continuous batching of LP solve requests on one GPU.
 *
 * A server keeps the active LPs of every attached handle (one sparse A each,
 * lpb.h) on the device; one worker thread per attached handle advances them
 * interval by interval: check_every iterations of the batched restarted Halpern PDHG
 * (Sec. 4-5 of the paper) followed by the FP64-accurate check.  Each request
 * -- a set of strong-branching children (Sec. 5.1) or bound-tightening LPs
 * (Sec. 5.2) of one matrix -- becomes one restart group: its LPs share the
 * batch-averaged restart test of Sec. 5 among themselves only, so a request
 * follows the same trajectory alone or among others.  Requests that arrive
 * while others run are admitted between intervals into free batch columns
 * of their matrix's lane, as long as the columns, restart groups and the
 * server's HBM budget allow; their iterations share the kernel launches of
 * the requests already running.  Handles run on their own CUDA streams, so
 * the intervals of different matrices overlap on the device.  A request that
 * stalls at FP32 resolution moves to the matrix's polish lane (double-float
 * or FP64 iterates per the handle's options).  Results stay on the device
 * until released, and a later request may start all of its LPs from one of
 * them (warm start from the parent's iterate, Sec. 5.1).
 *
 * All pointers are host pointers unless a name says _dev.  Inputs are
 * copied at submit.  Errors are return codes with lpb_last_error() set on
 * the calling thread; nothing aborts.
 */
#ifndef LPB_SERVE_H
#define LPB_SERVE_H

#include "lpb.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lpb_server* lpb_server_t;

typedef struct {
    int64_t hbm_budget_bytes;  /* device bytes the server may hold for lanes and request buffers;
                                  0 (default): 80% of the free device memory at create */
    int32_t lane_columns;      /* FP32 batch columns per attached matrix (default 256) */
    int32_t polish_columns;    /* polish-lane columns per attached matrix (default 64; 0: no polish lane) */
    int32_t max_groups;        /* concurrent requests per lane (default 64) */
    int32_t device;            /* CUDA device, or -1 for the current device */
} lpb_server_options;

typedef struct {
    int32_t matrix_id;         /* from lpb_server_attach */
    int32_t num_lps;           /* >= 1 and <= lane_columns */
    const lpb_lp_spec* specs;  /* num_lps override records (host, copied) */
    double tol;                /* relative KKT tolerance (> 0) */
    int64_t max_iter;          /* iteration cap, rounded up to a multiple of check_every */
    const double* warm_x;      /* n x num_lps column-major start (host, copied), or NULL */
    const double* warm_y;      /* m x num_lps, or NULL */
    int64_t warm_request;      /* >= 0: every LP starts from result warm_lp of this request, which
                                  must not be released; admission waits until it is done. -1: none */
    int32_t warm_lp;
} lpb_request;

typedef struct {
    int32_t state;             /* 0 pending, 1 running, 2 done, 3 failed */
    int32_t num_lps;
    int32_t optimal, infeasible, iteration_limit, other;  /* status counts once done */
    int64_t iters;             /* largest iteration count of its LPs */
    double t_submit, t_admit, t_done;  /* seconds since the server started */
    int64_t footprint_bytes;   /* device bytes charged to the budget while it is held */
    int32_t polished;          /* 1 if it moved to the polish lane */
} lpb_request_info;

typedef struct {
    int64_t submitted, done, lps_solved;  /* lps_solved: optimal or infeasible certificates */
    int64_t intervals;         /* lane intervals run */
    int64_t column_iters;      /* sum over intervals of active columns x iterations */
    int64_t admitted_while_busy;  /* requests admitted into a lane that had other work */
    int64_t migrations;        /* requests moved to a polish lane */
    double busy_s;             /* time during which some matrix had device work in flight */
    int64_t hbm_used_bytes, hbm_budget_bytes;
    int64_t kernels;           /* kernel launches of the intervals and checks */
} lpb_server_stats;

void lpb_server_default_options(lpb_server_options* opt);
lpb_err lpb_server_create(const lpb_server_options* opt, lpb_server_t* out);
/* Attaches a handle (created on the same device); the caller keeps ownership
 * but must not use it in lpb_solve while attached, nor destroy it before
 * the server.  Allocates the matrix's lanes from the budget. */
lpb_err lpb_server_attach(lpb_server_t srv, lpb_handle h, int32_t* matrix_id);
lpb_err lpb_server_submit(lpb_server_t srv, const lpb_request* req, int64_t* request_id);
/* *done = 1 once the request finished (or failed) */
lpb_err lpb_server_poll(lpb_server_t srv, int64_t request_id, int32_t* done);
/* Blocks until the request finished or timeout_s passed (LPB_ERR_TIMEOUT);
 * timeout_s < 0 waits without limit. */
lpb_err lpb_server_wait(lpb_server_t srv, int64_t request_id, double timeout_s);
/* results of a finished request: res for LP lp, and x (n), y (m) in the
 * original space if not NULL */
lpb_err lpb_server_result(lpb_server_t srv, int64_t request_id, int32_t lp, lpb_lp_result* res, double* x,
                          double* y);
lpb_err lpb_server_results(lpb_server_t srv, int64_t request_id, lpb_lp_result* res /* num_lps */);
lpb_err lpb_server_request_info(lpb_server_t srv, int64_t request_id, lpb_request_info* info);
/* frees a finished request's device results and returns its footprint */
lpb_err lpb_server_release(lpb_server_t srv, int64_t request_id);
lpb_err lpb_server_stats_get(lpb_server_t srv, lpb_server_stats* st);
/* stops the worker (requests still pending or running are dropped) and
 * frees everything the server allocated; attached handles stay valid */
void lpb_server_destroy(lpb_server_t srv);

#ifdef __cplusplus
}
#endif

#endif /* LPB_SERVE_H */
