"""Tile-shape autotuner of the batched sweep (lbs_batch_set_tiles).

The batched step runs its cell phases on tx x ty thread blocks and its SOR
rounds on one of three blocked tiles.  The best choice depends on the
lattice, the storage form and the channel widths: a tile wider than a narrow
channel idles threads on the walls' far side, a tall one loses the L1 reuse
of the stencils along x.  The tuner times candidates on the batch itself
(after a warm-up step, CUDA events on the batch's stream) by coordinate
search - the cell tile with SOR tile 0, then the SOR tile with the best
cell tile - and caches the winner by (lattice, storage, width class) in a
JSON file, so a later batch of the same class reuses it without timing.

Tile choice never changes results: the per-cell arithmetic and the SOR
iterates are independent of the decomposition.
"""
import json
import os

CELL_TILES = ((32, 8), (64, 4), (128, 2), (32, 4), (64, 2), (16, 16), (32, 16), (256, 1))
SOR_TILES = tuple(range(9))  # the variants of lbs_set_sor_tile
STORAGE_NAMES = {0: "f64", 1: "f32", 2: "f16", 3: "bf16"}


def width_class(widths):
    """Class of a batch by its typical channel width: the power of two at or
    above the median width (64, 128, 256, ...)."""
    ws = sorted(int(w) for w in widths)
    med = ws[len(ws) // 2]
    c = 32
    while c < med:
        c *= 2
    return f"w{c}"


def cache_key(lattice, storage, widths):
    st = STORAGE_NAMES.get(storage, storage) if isinstance(storage, int) else storage
    return f"{lattice}/{st}/{width_class(widths)}"


def default_cache_path():
    base = os.environ.get("LBS_TUNE_CACHE")
    if base:
        return base
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2311_15242_gb300",
                        "tiles.json")


def load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(path, cache):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def cuda_timer(batch, steps=2):
    """Milliseconds per step of `batch` (one warm-up step, then `steps`
    steps between CUDA events on its stream)."""
    import torch
    batch.step(1)
    batch.stream.synchronize()  # (instance statuses are left to the caller)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(batch.stream)
    batch.step(steps)
    b.record(batch.stream)
    b.synchronize()
    return a.elapsed_time(b) / steps


def tune(batch, widths, lattice="d2q9", timer=None, cache_path=None, use_cache=True,
         cell_tiles=CELL_TILES, sor_tiles=SOR_TILES):
    """Choose and apply the tile shapes of `batch` (anything with
    set_tiles(tx, ty, sor) and a `storage` attribute).  Returns a dict with
    the choice, where it came from ("cache" or "timed") and the timings.
    Note that timing advances the batch's state (warm-up and timed steps)."""
    timer = timer or cuda_timer
    path = cache_path or default_cache_path()
    key = cache_key(lattice, batch.storage, widths)
    cache = load_cache(path) if use_cache else {}
    if key in cache:
        c = cache[key]
        batch.set_tiles(c["tx"], c["ty"], c["sor"])
        return {"key": key, "source": "cache", **c}
    times = {}

    def run(tx, ty, sv):
        try:
            batch.set_tiles(tx, ty, sv)
        except RuntimeError:  # (a variant too large for this storage form)
            times[f"{tx}x{ty}/{sv}"] = float("inf")
            return float("inf")
        t = float(timer(batch))
        times[f"{tx}x{ty}/{sv}"] = t
        return t

    # 1. cell tile with the first SOR tile; 2. SOR tile with the best cell tile
    for tx, ty in cell_tiles:
        run(tx, ty, sor_tiles[0])
    tx, ty = min(cell_tiles, key=lambda t: times[f"{t[0]}x{t[1]}/{sor_tiles[0]}"])
    for v in sor_tiles:
        if f"{tx}x{ty}/{v}" not in times:
            run(tx, ty, v)
    sv = min(sor_tiles, key=lambda v: times[f"{tx}x{ty}/{v}"])
    choice = {"tx": tx, "ty": ty, "sor": sv, "ms_per_step": times[f"{tx}x{ty}/{sv}"]}
    batch.set_tiles(choice["tx"], choice["ty"], choice["sor"])
    if use_cache:
        cache = load_cache(path)
        cache[key] = choice
        save_cache(path, cache)
    return {"key": key, "source": "timed", "timings": times, **choice}


SOR_TILES_3D = (0, 1, 2, 3)  # red-black half-sweeps; z-marching full sweeps; column marching


def tune_single(solver, width, lattice="d2q9", timer=None, cache_path=None, use_cache=True,
                sor_tiles=None):
    """Choose and apply the SOR variant of a single context (anything with
    set_sor_tile(v) and a `storage` attribute): the blocked tiles in 2D, the
    two sweep forms in 3D; cached under the same width classes with the
    suffix /single."""
    if sor_tiles is None:
        sor_tiles = SOR_TILES_3D if lattice == "d3q19" else SOR_TILES
    timer = timer or cuda_timer
    path = cache_path or default_cache_path()
    key = cache_key(lattice, solver.storage, [width]) + "/single"
    cache = load_cache(path) if use_cache else {}
    if key in cache:
        solver.set_sor_tile(cache[key]["sor"])
        return {"key": key, "source": "cache", **cache[key]}
    times = {}
    for v in sor_tiles:
        try:
            solver.set_sor_tile(v)
        except RuntimeError:  # (a variant too large for this storage form)
            times[v] = float("inf")
            continue
        times[v] = float(timer(solver))
    sv = min(sor_tiles, key=lambda v: times[v])
    solver.set_sor_tile(sv)
    choice = {"sor": sv, "ms_per_step": times[sv]}
    if use_cache:
        cache = load_cache(path)
        cache[key] = choice
        save_cache(path, cache)
    return {"key": key, "source": "timed", "timings": {str(k): v for k, v in times.items()},
            **choice}
