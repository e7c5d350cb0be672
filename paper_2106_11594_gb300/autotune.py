"""Autotuner for the batched form. It picks two knobs by timing complete passes of the
caller's own batch on the GPU:
  * the per-block row cap (rg_batch_set_block_rows): the rows per internal block, Section
    3's block of observations;
  * in mixed mode, the tile grouping of the tensor-core projection's second product
    (rg_batch_set_tc_group): the 64-column slices issued per commit.

Each candidate pair is timed with CUDA events over `reps` full passes (reset, add_rows,
solution) after one untimed pass. The fastest pair is kept in the handle and returned with
the timings. Block caps above the capacity laid out at init are skipped. Results do not
depend on either knob; only the time does.
"""
from __future__ import annotations


def _pass_ms(bt, A_packed, row_offsets, elem_offsets, y_packed, X_packed, reps):
    import torch

    def one():
        bt.reset()
        bt.add_rows(A_packed, row_offsets, elem_offsets, y_packed)
        bt.solution(X_packed)

    one()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        one()
    t1.record()
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / reps


def tune(bt, A_packed, row_offsets, elem_offsets, y_packed, X_packed,
         block_rows=(64, 128, 256, 512), tc_groups=(2, 4, 6), reps: int = 1):
    """Grid search over (block row cap, tensor-core slice group). tc_groups=None keeps the
    group in force (FP64 batches, where it has no effect). Returns ({"block_rows": kb,
    "tc_group": g}, {"kb/g": ms})."""
    cap = bt.block_rows(0)
    g0 = bt.tc_group(0)
    groups = tuple(tc_groups) if tc_groups else (g0,)
    best, best_ms, times = None, float("inf"), {}
    for kb in block_rows:
        try:
            bt.block_rows(int(kb))
        except Exception:
            continue
        for g in groups:
            bt.tc_group(int(g))
            ms = _pass_ms(bt, A_packed, row_offsets, elem_offsets, y_packed, X_packed, reps)
            times[f"{int(kb)}/{int(g)}"] = ms
            if ms < best_ms:
                best, best_ms = (int(kb), int(g)), ms
    kb, g = best if best is not None else (cap, g0)
    bt.block_rows(kb)
    bt.tc_group(g)
    bt.sync()
    return {"block_rows": kb, "tc_group": g}, times


def tune_block_rows(bt, A_packed, row_offsets, elem_offsets, y_packed, X_packed,
                    candidates=(64, 128, 256, 512), reps: int = 1):
    """The block row cap alone (the slice group in force is kept). Returns (kb, {kb: ms})."""
    choice, times = tune(bt, A_packed, row_offsets, elem_offsets, y_packed, X_packed,
                         block_rows=candidates, tc_groups=None, reps=reps)
    return choice["block_rows"], {int(k.split("/")[0]): v for k, v in times.items()}
