"""Autotuning cache for the batched kernels (grom_autotune / grom_set_tuning).

A tuned entry depends on the ROM's shape and the device, so the cache is a
JSON file keyed by (form, storage, layout, n, rank, max_batch, SM count); each
key holds the entries autotune installed, one per batch bucket.  `apply`
re-installs them on a ROM of the same key in a later run, with no timing.

As a program it tunes synthetic ROMs of a given shape and writes the cache:

    python -m paper_2311_03694_gb300.tune --form full --layout skew_packed \\
        --n 512 --batches 16,64,256,1024 --out tune.json

Kernel times do not depend on the values, so the operators are plain seeded
normal draws (the full tensor made skew in its test and advected index,
as the skew-packed layout requires).
"""
import argparse
import json
import os

import numpy as np

from . import Rom, load


def key_of(rom, sm_count):
    return "%s/%s/%s/n%d/r%d/b%d/sm%d" % (rom.form, rom.storage, rom.layout, rom.n, rom.rank, rom.max_batch,
                                          sm_count)


def _read(path):
    if path and os.path.exists(path):
        with open(path) as fh:
            return json.load(fh)
    return {}


def tune(rom, batches, sm_count, reps=10, path=None):
    """Autotune `rom` for each batch size; returns the entries and, with
    `path`, merges them into that cache file."""
    entries = [rom.autotune(int(b), reps=reps) for b in batches]
    if path:
        cache = _read(path)
        cur = {e["batch"]: e for e in cache.get(key_of(rom, sm_count), [])}
        for e in entries:
            cur = {b: v for b, v in cur.items() if (b + 15) // 16 != (e["batch"] + 15) // 16}
            cur[e["batch"]] = e
        cache[key_of(rom, sm_count)] = [cur[b] for b in sorted(cur)]
        with open(path, "w") as fh:
            json.dump(cache, fh, indent=1, sort_keys=True)
    return entries


def apply(rom, sm_count, path):
    """Install the cached entries of the ROM's key; returns how many."""
    entries = _read(path).get(key_of(rom, sm_count), [])
    for e in entries:
        rom.set_tuning(e)
    return len(entries)


def _synthetic_rom(form, storage, layout, n, rank, max_batch, seed):
    rng = np.random.default_rng(seed)
    a = ((np.arange(1, n + 1) / n) ** 2).astype(np.float64)
    if form == "full":
        G = rng.standard_normal((n, n, n))
        C = G - G.transpose(2, 1, 0)
        del G
        return Rom(n, "full", storage, tensor=C, stiffness=a, max_batch=max_batch, layout=layout)
    facs = tuple(rng.standard_normal((n, rank)) / np.sqrt(rank) for _ in range(3))
    return Rom(n, form, storage, factors=facs, stiffness=a, max_batch=max_batch)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--form", default="full", choices=["full", "cp", "cp_skew"])
    ap.add_argument("--storage", default="bf16")
    ap.add_argument("--layout", default="dense", choices=["dense", "skew_packed"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--rank", type=int, default=0)
    ap.add_argument("--batches", default="16,64,256,1024")
    ap.add_argument("--max-batch", type=int, default=0, help="default: the largest of --batches")
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--seed", type=int, default=20231106)
    ap.add_argument("--out", default=None, help="cache file to merge the entries into")
    args = ap.parse_args(argv)
    import torch

    load()
    batches = [int(b) for b in args.batches.split(",")]
    sm = torch.cuda.get_device_properties(0).multi_processor_count
    rom = _synthetic_rom(args.form, args.storage, args.layout, args.n, args.rank,
                         args.max_batch or max(batches), args.seed)
    for e in tune(rom, batches, sm, reps=args.reps, path=args.out):
        print(json.dumps(dict(e, key=key_of(rom, sm), speedup=round(e["ms_rule"] / e["ms"], 4))))
    rom.close()


if __name__ == "__main__":
    main()
