"""Offline search of the batched form's level schedules over a workload.

The fields of a workload are grouped by shape class (ndim and ceil(log2)
of each extent, the key the schedule table uses) and configuration; for
each group one representative field runs the C-ABI search
(``hpez_tuning_search``: every candidate schedule timed on the GPU), and
the winners of every level and direction go into one table, saved as text.
The batched and served forms then read it with ``hpez_use_tuning``.

    python -m paper_2311_12133_gb300.autotune --out levels.txt

searches the 64-field benchmark mix (default and multi-dimensional
configurations) and writes the table.
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
    t = search_workload(ctx, mix_specs(a.fields), copies=a.copies, reps=a.reps, log=print,
                        save=a.out)
    t.save(a.out)
    print(f"{len(t)} entries -> {a.out}")
    ctx.close()


if __name__ == "__main__":
    main()
