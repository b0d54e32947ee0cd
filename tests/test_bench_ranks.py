"""The replica bookkeeping of bench.py (barrier, max over ranks, whole-job rate) with two
gloo ranks on the CPU: the path a torchrun --nproc-per-node 2 bench run takes."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks("gloo")
    r.barrier()
    t = r.max(1.0 + rank)                 # rank 1 is the slowest
    rate = r.total_rate(1000, t)
    r.barrier()
    q.put((rank, r.world, t, rate))
    r.close()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(i, 2, port, q)) for i in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, world, t, rate in out:
        assert world == 2
        assert t == 2.0                   # max over ranks
        assert rate == 2 * 1000 / 2.0     # all ranks' units / slowest time


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE"):
        os.environ.pop(k, None)
    r = bench.Ranks("gloo")
    assert r.world == 1 and r.max(3.5) == 3.5 and r.total_rate(10, 2.0) == 5.0


def _count_fold_apply(p):
    """Operations of one folded D contraction on a line of p nodes, counted loop by loop as
    the operator kernel runs them (FMA = 2 flops, add / subtract / multiply = 1)."""
    H, odd = p // 2, p % 2
    f = 2 * H                       # even / odd sums of the line
    for _ in range(H):
        f += 1 if odd else 0        # middle column times v[H]
        f += 2 * H + 2 * H          # the two H-term FMA chains
        f += 2                      # out[i] and out[n - i]
    if odd:
        f += 2 * H                  # the middle output
    return f


def _count_pencil(P):
    H, odd = P // 2, P % 2
    NE = P - H
    fwd = 2 * H
    for c in range(P):
        fwd += 2 * H + (1 if (odd and c < NE) else 0)
    bwd = 0
    for _ in range(H):
        bwd += 2 * NE + 2 * (P - NE) + 2
    if odd:
        bwd += 2 * NE
    return fwd, bwd


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_executed_flop_counts_follow_the_kernels(n):
    """bench.py's roofline counts equal the operations of the folded kernels, counted loop by
    loop: 6 p^2 operator lines and 19 flops per node (G grad u, the divergence sums and the
    lambda m u FMA); 3 P^2 forward and 3 P^2 backward pencil lines and P^3 diagonal scalings."""
    import bench
    p, P = n + 1, n + 3
    assert bench.ax_flops(n, 1) == 6 * p * p * _count_fold_apply(p) + 19 * p ** 3
    fwd, bwd = _count_pencil(P)
    assert bench.schwarz_flops(n, 1) == 3 * P * P * (fwd + bwd) + P ** 3
    # the folded forms cost less than the paper's unfolded counts
    assert bench.ax_flops(n, 1) < bench.ax_flops_paper(n, 1)
    assert bench.schwarz_flops(n, 1) < bench.schwarz_flops_paper(n, 1)


# FP32-pipe operations of the pair arithmetic (csrc/kdw.cuh): dw_add / dw_sub = TwoSum (6)
# + 2 adds, dw_mul = 1 multiply + 3 FMAs, dw_mac = dw_mul + TwoSum + 2 adds.
DW_ADD, DW_MUL, DW_MAC = 8, 4, 12


def _count_dw_fold(p):
    H, odd = p // 2, p % 2
    f = 2 * H * DW_ADD                  # even / odd sums of the line
    for _ in range(H):
        f += DW_MUL if odd else 0       # middle column times v[H]
        f += 2 * H * DW_MAC             # the two H-term accumulations
        f += 2 * DW_ADD                 # out[i] and out[n - i]
    if odd:
        f += H * DW_MAC                 # the middle output
    return f


def _count_dw_pencil(P):
    H, odd = P // 2, P % 2
    NE = P - H
    fwd = 2 * H * DW_ADD
    for c in range(P):
        fwd += H * DW_MAC + (DW_MUL if (odd and c < NE) else 0)
    bwd = 0
    for _ in range(H):
        bwd += (NE + (P - NE)) * DW_MAC + 2 * DW_ADD
    if odd:
        bwd += NE * DW_MAC
    return fwd, bwd


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6, 7, 8])
def test_pair_operation_counts_follow_the_kernels(n):
    """The double-FP32 rooflines count the FP32 operations of the pair kernels loop by loop:
    the same lines as the binary64 kernels with pair sums, products and multiply-accumulates;
    per operator node 3 metric rows (a product and two multiply-accumulates), the divergence
    sum, the lambda m u accumulate with its sum, one split and one join; per patch node one
    diagonal product and one split."""
    import bench
    p, P = n + 1, n + 3
    per_node = 3 * (DW_MUL + 2 * DW_MAC) + DW_ADD + (DW_ADD + DW_MAC) + 2 + 6
    assert bench.dw_ops_ax(n, 1) == 6 * p * p * _count_dw_fold(p) + per_node * p ** 3
    fwd, bwd = _count_dw_pencil(P)
    assert bench.dw_ops_schwarz(n, 1) == 3 * P * P * (fwd + bwd) + (DW_MUL + 2) * P ** 3


def _count_dw_metric():
    """geom_line_dw and geom_node_dw (csrc/kgeomdw.cuh) step by step: (per node, per line);
    dw_norm = one TwoSum (6), sign flips free, the reciprocal estimate on the special-function
    unit (not counted)."""
    TWO_SUM = 6
    # per line: hb, ha (a halving = 2 multiplies), ab (a product and a halving), the corner
    # sums (8 corners x 3 rows x 3 sums), renormalised U0, U1 (12) and J2 (3)
    line = 4 * 2 + 4 * (DW_MUL + 2) + 8 * 3 * 3 * DW_MAC + 15 * TWO_SUM
    # per node: J's first two columns (a product and a multiply-accumulate each, renormalised)
    node = 6 * (DW_MUL + DW_MAC + TWO_SUM)
    node += 9 * (DW_MUL + DW_MAC + TWO_SUM)      # cofactors, renormalised
    node += DW_MUL + 2 * DW_MAC                  # determinant
    # dw_div: renormalise y, q_h = x_h r, p = q_h y_h, its error by two FMAs, the remainder
    # (a pair difference), one sum and one product for q_l, a final TwoSum
    node += TWO_SUM + 1 + 1 + 2 + DW_ADD + 1 + 1 + TWO_SUM
    node += 6 * (DW_MUL + 2 * DW_MAC + DW_MUL)   # C^T C scaled by w / det
    node += DW_MUL                               # m
    return node, line


@pytest.mark.parametrize("n", [2, 5, 7, 8])
def test_recomputed_pair_operation_counts_follow_the_kernel(n):
    """The recomputed form: the same lines; per node the 3 metric rows, three divergence sums
    (the first adds to lambda m u instead of overwriting), lambda m u as two products, the
    split and the join, and the metric's per-node part; per line the metric's per-line part."""
    import bench
    p = n + 1
    node, line = _count_dw_metric()
    assert (node, line) == (580, 986)
    per_node = 3 * (DW_MUL + 2 * DW_MAC) + 3 * DW_ADD + 2 * DW_MUL + 2 + 6 + node
    assert bench.dw_ops_ax_recompute(n, 1) == 6 * p * p * _count_dw_fold(p) + per_node * p ** 3 + line * p * p
