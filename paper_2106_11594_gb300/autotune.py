"""Autotuner for the batched form: picks the per-block row cap (rg_batch_set_block_rows)
by timing complete passes of the caller's own batch on the GPU.

Each candidate is timed with CUDA events over `reps` full passes (reset, add_rows,
solution) after one untimed pass; the fastest candidate is kept in the handle and
returned with the timings. Candidates above the capacity laid out at init are skipped.
"""
from __future__ import annotations


def tune_block_rows(bt, A_packed, row_offsets, elem_offsets, y_packed, X_packed,
                    candidates=(64, 128, 256, 512), reps: int = 1):
    import torch

    cap = bt.block_rows(0)
    # the capacity is the largest value the library accepts; probe it
    best, best_ms, times = None, float("inf"), {}
    for kb in candidates:
        try:
            bt.block_rows(int(kb))
        except Exception:
            continue

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
        ms = t0.elapsed_time(t1) / reps
        times[int(kb)] = ms
        if ms < best_ms:
            best, best_ms = int(kb), ms
    bt.block_rows(best if best is not None else cap)
    bt.sync()
    return best, times
