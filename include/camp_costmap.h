/*
 * camp_costmap.h -- C ABI of the actor's cost map (Sec. V-A; Sec. III-C: the
 * actor maps an observation to the stage-cost parameters of the MPC layer),
 * run on the tensor cores of GB300 (sm_103a).
 *
 * The map is an MLP with two hidden layers of `hidden` (512 in Sec. V-A) ReLU
 * units and a sigmoid output layer scaled to the cost weights' bounds:
 *
 *     o   = [x_init; x_ref,0]                       (26 values per instance)
 *     h1  = relu(o W1 + b1),  h2 = relu(h1 W2 + b2)
 *     Q   = q_lo + (q_hi - q_lo) sigmoid(h2 W3 + b3)  (N * 13 values: Q_t per stage)
 *
 * Q is written as [B, N, 13], the layout of mpc_problem.Q with Nq = N, so the
 * forward can write straight into the buffer a following mpc_solve_fwd reads.
 * The backward takes dL/dQ (the layer's mpc_solve_bwd output) back through
 * the three layers to dL/dW_l, dL/db_l and optionally dL/do.
 *
 * Conventions: every pointer is a device pointer on the current device, row-
 * major FP32; W_l is [n_in_l, n_out_l] (W1 [26, hidden], W2 [hidden, hidden],
 * W3 [hidden, N * 13]).  The caller owns all buffers, including the workspace
 * of mpc_costmap_workspace_bytes(B, hidden, n_out) bytes (256-byte aligned),
 * which keeps the activations the backward needs: mpc_costmap_backward must
 * get the workspace of the matching mpc_costmap_forward, unchanged since.
 * The calls allocate nothing and do not synchronise (capturable in a CUDA
 * graph); return codes come from host validation and the launches.  Every
 * device wait is bounded: the int at the start of the workspace is set
 * nonzero when one gave up (the results are then invalid), and cleared by
 * each forward.  A workspace sized for B_max serves every B <= B_max.
 */
#ifndef CAMP_COSTMAP_H
#define CAMP_COSTMAP_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mpc_costmap {
    int          n_in;              /* 26: [x_init; x_ref,0]                          */
    int          hidden;            /* units per hidden layer (512 in Sec. V-A)       */
    int          n_out;             /* N * 13: Q_t of every stage                      */
    const float *W1, *b1;           /* [26, hidden], [hidden]                          */
    const float *W2, *b2;           /* [hidden, hidden], [hidden]                      */
    const float *W3, *b3;           /* [hidden, n_out], [n_out]                        */
    float        q_lo, q_hi;        /* bounds of the weights, q_lo < q_hi              */
} mpc_costmap;

/* Workspace bytes for a batch of B (0 for invalid sizes). */
size_t mpc_costmap_workspace_bytes(int B, int hidden, int n_out);

/* Q [B, N, 13] from x_init [B, 13] and x_ref [B, N, 13] (its stage 0 enters
 * the observation).  Errors: MPC_ERR_ARG (NULL pointer, q_hi <= q_lo),
 * MPC_ERR_SHAPE (n_in != 26, n_out != N * 13, B < 0), MPC_ERR_CUDA. */
int mpc_costmap_forward(const mpc_costmap *net, int B, int N, const float *x0, const float *x_ref, float *Q,
                        void *ws, cudaStream_t stream);

/* dL/dW1 [26, hidden], dL/db1, dL/dW2, dL/db2, dL/dW3, dL/db3 (sums over the
 * batch) and, when d_obs is not NULL, dL/do [B, 26], from dL/dQ [B, N, 13].
 * Same errors as the forward. */
int mpc_costmap_backward(const mpc_costmap *net, int B, int N, const float *x0, const float *x_ref,
                         const float *dQ, void *ws, float *dW1, float *db1, float *dW2, float *db2, float *dW3,
                         float *db3, float *d_obs, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CAMP_COSTMAP_H */
