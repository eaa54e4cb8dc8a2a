"""Offline search of the batched form's level schedules over a workload.

The fields of a workload are grouped by shape class (ndim and the
half-octave floor(2 log2 n) of each extent, the key the schedule table uses) and configuration; for
each group one representative field runs the C-ABI search
(``hpez_tuning_search``: every candidate schedule timed on the GPU), and
the winners of every level and direction go into one table, saved as text.
The batched and served forms then read it with ``hpez_use_tuning``.

    python -m paper_2311_12133_gb300.autotune --out levels.txt

searches the 64-field benchmark mix (default and multi-dimensional
configurations) and the benchmark's single fields (with the tuner's
configuration where they are auto-tuned), and writes the table.
"""
import argparse
import os

from . import fields, hpez

SHIPPED = os.path.join(os.path.dirname(__file__), "tuning", "levels_gb300.txt")


def class_of(shape, cfg_kw):
    """The group a field falls in: its level-1 key without the direction,
    and its configuration."""
    cfg = hpez.make_config(len(shape), **cfg_kw) if cfg_kw else None
    key = hpez.hpez_level_key_of(tuple(shape), cfg, 1, False)
    return key[:4], tuple(sorted((cfg_kw or {}).items()))


def search_workload(ctx, specs, copies=0, reps=3, tuning=None, log=None, save=None):
    """specs: (kind, shape, seed, rel eb, config kwargs or None) per field.
    Returns the table (a new one unless `tuning` is given); with `save`, the
    table is written there after every class."""
    t = tuning if tuning is not None else hpez.Tuning()
    seen = set()
    for kind, shape, seed, eb, kw in specs:
        c = class_of(shape, kw)
        if c in seen:
            continue
        seen.add(c)
        x = fields.make_torch(kind, shape, seed)
        cfg = hpez.make_config(len(shape), **kw) if kw else None
        t.search(ctx, x, eb, hpez.HPEZ_EB_REL, cfg, copies=copies, reps=reps)
        del x
        if save:
            t.save(save)
        if log:
            log(f"searched class {c[0]} {dict(c[1])}: {len(t)} entries", flush=True)
    return t


# single fields of the benchmark set: (generator, shape, configuration)
# with "tuned" = the Sec. 6 tuner's choice for the field
# in order of importance: where two fields share a shape class (and a
# level's interpolator and paradigm), the earlier one's entries are kept
WORKLOADS = [
    ("grf", (512, 512, 512), "tuned"),
    ("lognormal", (512, 512, 512), "tuned"),
    ("grf", (100, 500, 500), "tuned"),
    ("bumps", (128, 128, 128), None),
    ("aniso", (98, 1200, 1200), "tuned"),
    ("aniso", (98, 1200, 1200), {"paradigm": 1, "interp": 1}),
    ("aniso", (98, 1200, 1200), {"interp": 1, "same_level": 1}),
    ("climate2d", (1800, 3600), "tuned"),
    ("climate2d", (1800, 3600), {"paradigm": 1, "interp": 1}),
    ("climate2d", (1800, 3600), {"interp": 1, "same_level": 1}),
]


def merge_first_wins(tables):
    """One table from several, in order of importance: an entry comes from
    the first table that holds its key."""
    import tempfile
    out = hpez.Tuning()
    with tempfile.TemporaryDirectory() as d:
        for i, t in enumerate(reversed(tables)):
            path = os.path.join(d, f"t{i}.txt")
            t.save(path)
            out.load(path)  # later loads replace earlier entries
    return out


def search_fields(ctx, workloads=WORKLOADS, eb=1e-3, reps=3, tuning=None, log=None,
                  save=None):
    """The search for each single field (one copy per batch when the field
    holds 2^25 points or more): the tuner's configuration where the
    workload says "tuned".  Fields earlier in `workloads` keep their
    entries where later ones share a key."""
    import torch
    done = [tuning] if tuning is not None else []
    for kind, shape, how in workloads:
        x = fields.make_torch(kind, shape, fields.seed_of("autotune", kind, *shape))
        if how == "tuned":
            cfg, _ = hpez.hpez_tune(ctx.handle, x.data_ptr(), shape, hpez.HPEZ_EB_REL, eb, None,
                                    torch.cuda.current_stream().cuda_stream)
        else:
            cfg = hpez.make_config(len(shape), **how) if how else None
        t = hpez.Tuning()
        t.search(ctx, x, eb, hpez.HPEZ_EB_REL, cfg, copies=0, reps=reps)
        del x
        torch.cuda.empty_cache()
        done.append(t)
        if save:
            merge_first_wins(done).save(save)
        if log:
            log(f"searched {kind} {shape} {how}: {len(t)} entries", flush=True)
    return merge_first_wins(done)


def mix_specs(n_fields=64, seed=0, configs=(None, {"paradigm": 1, "interp": 0})):
    """The benchmark mix under each configuration."""
    out = []
    for kw in configs:
        for kind, shape, sd, eb in fields.batch_mix(n_fields, seed=seed):
            out.append((kind, shape, sd, eb, kw))
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--out", default=SHIPPED)
    ap.add_argument("--fields", type=int, default=64)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--copies", type=int, default=0)
    a = ap.parse_args()
    ctx = hpez.Context(0)
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    # the benchmark's single fields first (their entries win), then the
    # classes of the 64-field mix that they leave open
    t = search_fields(ctx, reps=a.reps, log=print, save=a.out)
    m = search_workload(ctx, mix_specs(a.fields), copies=a.copies, reps=a.reps, log=print)
    t = merge_first_wins([t, m])
    t.save(a.out)
    print(f"{len(t)} entries -> {a.out}")
    ctx.close()


if __name__ == "__main__":
    main()
