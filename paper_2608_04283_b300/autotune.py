"""Launch-shape autotuner for the step kernel.

For a system, precision and grid side it times the step kernel over candidate
tiles (cells along x per block x rows per block) and both kernel variants
(plain loads; bulk-copy row pipeline with 2 to 4 stages) with CUDA events on the
simulation's stream, after warm-up, on a synthetic state of that size, and
records the fastest in tuning.json (looked up by bench.py and the server by the
nearest side).  Usage (GPU):
    python -m paper_2608_04283_b300.autotune euler fp32 1024 [--write]
"""
from __future__ import annotations

import argparse
import json
import os

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")
# (tx, -1): the height that fills whole waves of resident blocks
TILES = [(32, 8), (32, 16), (64, 4), (64, 8), (64, 16), (64, 32), (128, 4), (128, 8), (128, 16), (128, 32),
         (128, 64), (256, 4), (256, 8), (64, -1), (128, -1), (256, -1)]
VARIANTS = [(0, 0), (1, 2), (1, 3), (1, 4)]


def _state(system, n):
    if system == "euler":
        return inputs.isentropic_vortex(n), dict(omega=2.0, cfl=0.3, gamma=1.4), 10.0
    if system == "mhd_glm":
        return inputs.orszag_tang(n), dict(omega=1.0, cfl=0.3, gamma=5.0 / 3.0), 2 * np.pi
    return inputs.swe_hump_2d(n, 0.5, 0.5, 0.5, 0.08), dict(omega=1.0, cfl=0.3), 1.0


def tune(system, precision, n, steps=30, warmup=5, tiles=TILES, variants=VARIANTS):
    import torch
    from . import vklb
    U0, kw, L = _state(system, n)
    stream = torch.cuda.Stream()
    sim = vklb.Sim(system, (n, n), (0, 0), (L, L), precision=precision, stream=stream, **kw)
    U0d = torch.from_numpy(U0).cuda()
    results = []
    for var in variants:
        for tile in tiles:
            try:
                sim.set_tiling(64, 8)      # a shape every variant accepts
                sim.set_variant(*var)
                sim.set_tiling(*tile)      # the wave-fit height depends on the variant
            except vklb.VKLBError:
                continue
            sim.set_state(U0d)
            sim.step(warmup)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            e1.synchronize()
            sim.sync()
            results.append({"variant": list(var), "tile": list(tile), "ms": e0.elapsed_time(e1) / steps,
                            "resolved": [sim.info.tile_x, sim.info.tile_y], "blocks_per_sm": sim.info.blocks_per_sm})
    sim.close()
    results.sort(key=lambda r: r["ms"])
    return results


def write(system, precision, n, best):
    tab = json.load(open(TABLE))
    ent = tab.setdefault(f"{system}/{precision}", {})
    ent[str(n)] = best["tile"]
    var = tab.setdefault("_variants", {})
    if best["variant"][0] != 0:
        var[f"{system}/{precision}/{n}"] = best["variant"]
    else:
        var.pop(f"{system}/{precision}/{n}", None)
    json.dump(tab, open(TABLE, "w"), indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("system")
    ap.add_argument("precision")
    ap.add_argument("n", type=int)
    ap.add_argument("--write", action="store_true")
    a = ap.parse_args()
    res = tune(a.system, a.precision, a.n)
    for r in res[:8]:
        print(json.dumps(r))
    if a.write and res:
        write(a.system, a.precision, a.n, res[0])


if __name__ == "__main__":
    main()
