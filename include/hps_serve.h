/*
 * hps_serve.h -- request server on top of the HPS solver (include/hps.h).
 *
 * The paper solves one problem at a time and remarks (Section 5.2, forward
 * scattering) that once the operators are built, further sources cost only
 * a few more matrix-vector products and can be solved in parallel.  This
 * server (no counterpart in the paper) keeps built operators resident on one
 * GPU and answers a stream of requests against them:
 *   - solve requests (g, and optionally a new f) on a resident operator;
 *   - build requests that (re)build the operator of a slot from new
 *     coefficients, admitted only when the server's device-memory budget
 *     (hps_plan_bytes) has room.
 * Solve requests that wait on the same operator are merged into one batched
 * solve of up to max_batch right-hand sides; apply-only requests (the
 * build-time source) waiting on up to max_group different operators --
 * whatever their depths, orders and kinds -- are served together by one
 * hps_solve_multi, whose downward passes share launches level by level;
 * batches run concurrently on n_streams CUDA streams; builds
 * run on n_builders host threads, each with its own stream, while solves
 * continue.  Requests
 * that arrive while others run are admitted as soon as a stream and the
 * operator are free (continuous batching).  Requests on one slot take effect
 * in submission order: a solve submitted after a build of its slot uses the
 * new operator.
 *
 * Buffers: g, f, u of solves and every array of a build are host memory
 * (pageable is fine) owned by the caller, who keeps them valid and untouched
 * until the request's ticket has completed (hps_server_wait or a poll that
 * does not return HPS_PENDING).
 *
 * Threads: the server runs a scheduler thread and n_builders builder threads.  The
 * submit, wait and poll calls may be made from any thread.  Operators'
 * handles belong to the server.
 */
#ifndef HPS_GB300_SERVE_H
#define HPS_GB300_SERVE_H

#include "hps.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hps_server hps_server;

typedef struct {
  int version;          /* 1 */
  int n_slots;          /* operator slots 0..n_slots-1 (1..1024; 0 -> 16)            */
  int n_streams;        /* concurrent solve batches on the device (1..64; 0 -> 4)     */
  int max_batch;        /* right-hand sides merged into one batched solve (1..256;
                           0 -> 8)                                                  */
  int64_t hbm_budget;   /* device bytes the operators may hold; 0 -> 85 % of the free
                           device memory when the server is created                  */
  int lazy_root;        /* build operators with hps_options.lazy_root when the build
                           request passes no options                                 */
  int n_builders;       /* builds that may run at once, each on its own host thread
                           and stream (1..8; 0 -> 2)                                 */
  int max_group;        /* operators whose apply-only solves (build-time source) are
                           served by one hps_solve_multi: their downward passes
                           share launches across depths, orders and kinds
                           (1..24; 0 -> 8; 1 turns cross-operator batching off)    */
  int reserved[5];
} hps_server_options;

typedef struct {
  int status;           /* HPS_OK or the request's error                             */
  int kind;             /* 0 solve, 1 build                                           */
  int slot;
  int batch;            /* right-hand sides in the batched solve it ran in (solves)   */
  double t_submit_ms;   /* host clock, ms since the server was created                */
  double t_start_ms;    /* when its work was enqueued (solves) or started (builds)    */
  double t_done_ms;     /* when the server saw it finish (results in place)          */
} hps_ticket_info;

typedef struct {
  int64_t solves, builds, batches;  /* completed                                       */
  int64_t max_batch_seen;           /* requests in one dispatched batch                */
  int64_t multi_batches;            /* batches that served more than one operator      */
  int64_t max_group_seen;           /* operators in one dispatched batch               */
  int64_t resident_bytes;           /* device bytes of the resident operators          */
  int64_t hbm_budget;
} hps_server_stats;

/* Create a server on the calling thread's current CUDA device.  opts may be
 * NULL.  HPS_ERR_INVALID for out-of-range options, HPS_ERR_CUDA. */
hps_status hps_server_create(const hps_server_options* opts, hps_server** out);

/* Finish every submitted request, then release operators, streams and
 * buffers.  NULL is accepted. */
void hps_server_destroy(hps_server* s);

/* (Re)build the operator of `slot` (uniform trees; the same arguments as
 * hps_build).  opts may be NULL.  The request fails with HPS_ERR_OOM when the
 * planned footprint does not fit the budget even after the slot's old
 * operator is released. */
hps_status hps_server_submit_build(hps_server* s, int slot, const hps_tree* tree, int p, int q,
                                   const hps_coeffs* coeffs, const void* f, const hps_options* opts,
                                   int64_t* ticket);

/* Solve on the operator of `slot`: g [n_root_bdry], f NULL (the build-time
 * source) or [n_leaves][p^d], u [n_leaves][p^d] (dtype of the operator).
 * The request fails with HPS_ERR_INVALID if the slot holds no operator when
 * its turn comes. */
hps_status hps_server_submit_solve(hps_server* s, int slot, const void* g, const void* f, void* u,
                                   int64_t* ticket);

/* Block until the request has finished, fill *info (may be NULL) and release
 * the ticket.  Returns the request's status; HPS_ERR_INVALID for an unknown
 * ticket. */
hps_status hps_server_wait(hps_server* s, int64_t ticket, hps_ticket_info* info);

/* HPS_PENDING while the request runs; otherwise as hps_server_wait. */
hps_status hps_server_poll(hps_server* s, int64_t ticket, hps_ticket_info* info);

/* Counters (a consistent snapshot). */
hps_status hps_server_get_stats(hps_server* s, hps_server_stats* out);

/* The operator of a slot, for inspection once every request on that slot
 * has completed (NULL if none); valid until the slot's next build or the
 * server's destruction.  It must not be used while requests on the slot run. */
hps_status hps_server_operator(hps_server* s, int slot, hps_handle** h);

#ifdef __cplusplus
}
#endif

#endif /* HPS_GB300_SERVE_H */
