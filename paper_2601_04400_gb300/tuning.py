"""Autotuners of the fused stage kernel's tile shape and of the batched launches.

Every variant computes identical results; only speed differs.  `autotune` times a few
js_step calls per variant with CUDA events on the solver's stream, selects the fastest and
caches the choice in a JSON file keyed by grid size, physics and immersed body, so later
solvers with the same key start tuned.
"""
import json
import os

_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tuning.json")


def _key(solver):
    sp = solver._spec
    return "%dx%d|visc=%d|av=%d|ib=%d" % (sp["nx"], sp["ny"], int(sp["mu"] > 0), int(sp["nu"] > 0),
                                          int(getattr(solver, "has_ib", False)))


def _load():
    try:
        with open(_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(cache):
    os.makedirs(os.path.dirname(_CACHE), exist_ok=True)
    tmp = _CACHE + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, _CACHE)


def cached_variant(solver):
    return _load().get(_key(solver), {}).get("variant")


def apply_cached(solver):
    v = cached_variant(solver)
    if v is not None:
        solver.set_tuning(v)
    return v


def autotune(solver, U, reps=3, use_cache=True):
    """Time every stage-kernel variant on state U (not modified) and select the fastest.
    Returns {variant: ms per step}."""
    import torch
    if use_cache and apply_cached(solver) is not None:
        return {}
    dt = 0.5 * solver.max_dt(U, 0.5)
    _, n = solver.tuning()
    stream = torch.cuda.current_stream()
    times = {}
    work = U.clone()
    for v in range(n):
        solver.set_tuning(v)
        solver.step(work, dt, 1)  # warm-up (first launch sets kernel attributes)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            solver.step(work, dt, 1)
        t1.record(stream)
        t1.synchronize()
        times[v] = t0.elapsed_time(t1) / reps
        work.copy_(U)
    # keep the default (TMA-staged) variant unless another is clearly faster
    best = min(times, key=times.get)
    if times[best] > 0.98 * times[0]:
        best = 0
    solver.set_tuning(best)
    cache = _load()
    cache[_key(solver)] = {"variant": best, "ms_per_step": times}
    _save(cache)
    return times


# ---------------------------------------------------------------------------------------
# batched path: blocks per SM and tile schedule of the persistent forward launch
# ---------------------------------------------------------------------------------------
def batch_key(problems):
    """The instance mix: grid sizes, physics and immersed bodies of all instances (order-free)."""
    import hashlib
    items = sorted("%dx%d|visc=%d|av=%d|ib=%d" % (p.nx, p.ny, int(p.mu > 0), int(p.nu > 0), int(p.sdf is not None))
                   for p in problems)
    return "batch|%d|%s" % (len(items), hashlib.sha1("\n".join(items).encode()).hexdigest()[:16])


def autotune_batch(batch, problems, states, steps=2, use_cache=True):
    """Time js_batch_step for every (blocks per SM, schedule) on copies of `states` (which are
    not advanced) and select the fastest; the choice is cached per instance mix.  Results are
    identical for every choice.  The batch's registered states are `states` afterwards.
    Returns {(blocks_per_sm, schedule): ms per step} ({} when the cache had the choice)."""
    import torch
    key = batch_key(problems)
    cache = _load()
    if use_cache and key in cache:
        batch.set_tuning(*cache[key]["choice"])
        batch.set_states(states)
        return {}
    _, most, _, nsched = batch.tuning()
    work = [U.clone() for U in states]
    batch.set_states(work)
    stream = torch.cuda.current_stream()
    times = {}
    for bps in range(1, most + 1):
        for sched in range(nsched):
            batch.set_tuning(bps, sched)
            for U, U0 in zip(work, states):
                U.copy_(U0)
            batch.step(0.5, 1)  # warm-up
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            batch.step(0.5, steps)
            t1.record(stream)
            t1.synchronize()
            times[(bps, sched)] = t0.elapsed_time(t1) / steps
    if batch.status() != 0:
        raise RuntimeError("batched tuning run failed")
    default = (most, 0)
    best = min(times, key=times.get)
    if times[best] > 0.98 * times[default]:
        best = default
    batch.set_tuning(*best)
    batch.set_states(states)
    cache = _load()
    cache[key] = {"choice": list(best), "ms_per_step": {"%d,%d" % k: v for k, v in times.items()}}
    _save(cache)
    return times


def autotune_batch_reverse(batch, problems, states, dts, reps=2, use_cache=True):
    """Time js_batch_step_vjp (one reverse step of every instance from `states` with step sizes
    `dts`) in both launch forms -- one persistent launch, one launch per phase -- and select the
    faster; the choice is cached per instance mix.  Results are identical for both forms.
    Returns {split: ms per reverse step} ({} when the cache had the choice)."""
    import torch
    key = batch_key(problems) + "|reverse"
    cache = _load()
    if use_cache and key in cache:
        batch.set_reverse_launch(cache[key]["split"])
        return {}
    lam = [torch.randn_like(U) for U in states]
    out = [torch.empty_like(U) for U in states]
    stream = torch.cuda.current_stream()
    times = {}
    for split in (0, 1):
        batch.set_reverse_launch(split)
        batch.step_vjp(states, dts, lam, out)  # warm-up (the first call prepares the workspace)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(reps):
            batch.step_vjp(states, dts, lam, out)
        t1.record(stream)
        t1.synchronize()
        times[split] = t0.elapsed_time(t1) / reps
    if batch.status() != 0:
        raise RuntimeError("batched reverse tuning run failed")
    best = 1 if times[1] < 0.98 * times[0] else 0
    batch.set_reverse_launch(best)
    cache = _load()
    cache[key] = {"split": best, "ms_per_reverse_step": {str(k): v for k, v in times.items()}}
    _save(cache)
    return times
