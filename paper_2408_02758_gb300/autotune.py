"""Autotuner for the launch shapes of the FTLE kernels.

Candidates (threads per block, resident blocks per SM, gradient tile) are timed on the caller's
own problem through the C-ABI with CUDA events, and the fastest is kept in a JSON cache keyed by
GPU name, kernel and a shape bucket (dimension, flow kind, precision, log2 of the node count,
log2 of the step count).  The tuner only picks among launch shapes: every candidate computes the
same per-node arithmetic, so results do not depend on the choice.

    opts = autotune.options_for_compute(dm, flow, T, dt, "fp32c")   # ftle_options
    out = ftle.compute(dm, flow, T, dt, "fp32c", options=opts)
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass
from pathlib import Path
from typing import Callable, Iterable

ADVECT_CANDIDATES = [(256, 32), (256, 8), (128, 16), (64, 32), (256, 4), (128, 64)]
# gradient: the staged kernels (fixed-width list or CSR rows, fixed 256-thread tiles; the plain
# kernels where they do not apply) or plain loads with 128 / 256 threads per block
GRAD_CANDIDATES = [{"grad_staging": 0}, {"grad_block": 128, "grad_staging": 1}, {"grad_block": 256, "grad_staging": 1}]
BATCH_TILE_CANDIDATES = [(256, 256), (128, 512), (256, 1024), (64, 256)]


def cache_path() -> Path:
    base = os.environ.get("FTLE_AUTOTUNE_CACHE")
    if base:
        return Path(base)
    root = Path(os.environ.get("XDG_CACHE_HOME", Path.home() / ".cache"))
    return root / "ftle_gb300" / "autotune.json"


@dataclass
class Choice:
    params: dict
    ms: float


class Cache:
    def __init__(self, path: Path | None = None):
        self.path = Path(path) if path else cache_path()
        self.data = {}
        if self.path.exists():
            try:
                self.data = json.loads(self.path.read_text())
            except (OSError, ValueError):
                self.data = {}

    def get(self, key: str):
        v = self.data.get(key)
        return Choice(v["params"], v["ms"]) if v else None

    def put(self, key: str, choice: Choice):
        self.data[key] = {"params": choice.params, "ms": choice.ms}
        try:
            self.path.parent.mkdir(parents=True, exist_ok=True)
            tmp = self.path.with_suffix(".tmp")
            tmp.write_text(json.dumps(self.data, indent=1, sort_keys=True))
            os.replace(tmp, self.path)
        except OSError:
            pass  # a read-only cache location only costs re-tuning


def shape_key(gpu: str, kernel: str, dim: int, kind: int, precision: str, n_nodes: int, n_steps: int) -> str:
    nb = int(math.log2(max(1, n_nodes)))
    sb = int(math.log2(max(1, n_steps)))
    return f"{gpu}|{kernel}|d{dim}|k{kind}|{precision}|n2^{nb}|s2^{sb}"


def pick(candidates: Iterable[dict], timer: Callable[[dict], float], repeats: int = 2) -> Choice:
    """Time every candidate (best of `repeats`) and return the fastest; candidates that fail are
    skipped."""
    best = None
    for c in candidates:
        try:
            t = min(timer(c) for _ in range(repeats))
        except Exception:
            continue
        if best is None or t < best.ms:
            best = Choice(dict(c), float(t))
    if best is None:
        raise RuntimeError("autotune: every candidate failed")
    return best


def _gpu_name() -> str:
    import torch

    return torch.cuda.get_device_name()


def _event_timer(fn: Callable[[], None]) -> float:
    import torch

    s = torch.cuda.current_stream()
    fn()  # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def options_for_compute(mesh, flow, T: float, dt: float, precision: str = "fp32c", cache: Cache | None = None,
                        retune: bool = False):
    """ftle_options with the fastest advection block shape and gradient block for this problem."""
    from . import ftle

    return ftle.make_options(**params_for_compute(mesh, flow, T, dt, precision, cache, retune))


def params_for_compute(mesh, flow, T: float, dt: float, precision: str = "fp32c", cache: Cache | None = None,
                       retune: bool = False) -> dict:
    """The launch shapes options_for_compute picks, as ftle.make_options keyword arguments."""
    from . import ftle

    cache = cache or Cache()
    n_steps = int(round(abs(T) / dt))
    layout = "stencil" if mesh.desc.stencil else ("ell" if mesh.desc.ell_width else "csr")
    key = shape_key(_gpu_name(), f"compute-{layout}", mesh.dim, int(flow.kind), precision, mesh.n_nodes, n_steps)
    ch = None if retune else cache.get(key)
    if ch is None:
        phi = ftle.flowmap_empty(mesh.dim, mesh.n_nodes, precision)

        def t_adv(c):
            o = ftle.make_options(advect_block=c["advect_block"], advect_blocks_per_sm=c["advect_blocks_per_sm"])
            return _event_timer(lambda: ftle.ftle_advect(mesh, flow, 0.0, T, dt, precision, phi, options=o))

        adv = pick([{"advect_block": b, "advect_blocks_per_sm": s} for b, s in ADVECT_CANDIDATES], t_adv)

        gr = _pick_gradient(mesh, phi, precision, T)  # phi: the last advection's flowmap
        ch = Choice({**adv.params, **gr.params}, adv.ms + gr.ms)
        cache.put(key, ch)
    return dict(ch.params)


def _pick_gradient(mesh, phi, precision: str, T: float) -> Choice:
    from . import ftle

    out = ftle.ftle_out_empty(mesh.n_nodes, precision)
    ws = ftle.workspace_empty(ftle.ftle_workspace_bytes(mesh.n_nodes))

    def t_grad(c):
        o = ftle.make_options(**c)
        return _event_timer(lambda: ftle.ftle_gradient_eig(mesh, phi, precision, T, out, None, ws, options=o))

    return pick(GRAD_CANDIDATES, t_grad)


def params_for_gradient(mesh, phi, precision: str, T: float, cache: Cache | None = None,
                        retune: bool = False) -> dict:
    """The gradient launch shape (block, index staging) alone, for this mesh's neighbour layout,
    timed on the flowmap phi; as ftle.make_options keyword arguments."""
    cache = cache or Cache()
    layout = "stencil" if mesh.desc.stencil else ("ell" if mesh.desc.ell_width else "csr")
    key = shape_key(_gpu_name(), f"gradient-{layout}", mesh.dim, 0, precision, mesh.n_nodes, 1)
    ch = None if retune else cache.get(key)
    if ch is None:
        ch = _pick_gradient(mesh, phi, precision, T)
        cache.put(key, ch)
    return dict(ch.params)


def options_for_batch(meshes, flows, T, dt: float, precision: str = "fp32c", cache: Cache | None = None,
                      retune: bool = False):
    """ftle_options (advection block, gradient tile) with the fastest batched launch sequence."""
    from . import ftle

    return ftle.make_options(**params_for_batch(meshes, flows, T, dt, precision, cache, retune))


def params_for_batch(meshes, flows, T, dt: float, precision: str = "fp32c", cache: Cache | None = None,
                     retune: bool = False) -> dict:
    """The launch shapes options_for_batch picks, as ftle.make_options keyword arguments."""
    from . import ftle

    cache = cache or Cache()
    n = sum(m.n_nodes for m in meshes)
    steps = max(int(round(abs(t) / dt)) for t in T)
    key = shape_key(_gpu_name(), f"batch{len(meshes)}", meshes[0].dim, int(flows[0].kind), precision, n, steps)
    ch = None if retune else cache.get(key)
    if ch is None:
        import torch

        outs = [torch.empty(m.n_nodes, dtype=torch.float32, device="cuda") for m in meshes]
        ws = ftle.workspace_empty(ftle.ftle_batch_workspace_bytes(meshes, precision))

        def t_batch(c):
            o = ftle.make_options(advect_block=c["advect_block"], grad_tile=c["grad_tile"])
            return _event_timer(lambda: ftle.ftle_batch(meshes, flows, T, dt, precision, outs, ws, options=o))

        ch = pick([{"advect_block": b, "grad_tile": t} for b, t in BATCH_TILE_CANDIDATES], t_batch, repeats=1)
        cache.put(key, ch)
    return {k: v for k, v in ch.params.items() if k in ("advect_block", "grad_tile")}
