"""The five benchmark workloads: model sizes, seeds and system recipes.

Seeds: systems 20260202 + workload index, weights 1234, velocities 42.
Model dimensions are plain numbers; the arithmetic lives elsewhere.
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

from . import System, cached, protein_in_water, water_box

SYSTEM_SEED = 20260202
WEIGHT_SEED = 1234
VELOCITY_SEED = 42


@dataclass(frozen=True)
class AttnModel:
    """Attention-family sizes: embedding 1->e1->e2->m1, axis m2, L layers."""
    n_species: int
    e1: int
    e2: int
    m1: int
    m2: int
    n_layers: int
    hidden: int
    heads: int
    f1: int
    f2: int
    f3: int
    nmax: int
    rc: float = 6.0
    rs: float = 0.5
    fit_heads: int = 1
    message_passing: int = 0     # 1: atom channel passed between neighbours each layer

    def as_dict(self):
        return asdict(self)


@dataclass(frozen=True)
class GraphModel:
    """Graph-family sizes: node dim, edge dim, L layers, angle cutoff/limit."""
    n_species: int
    node: int
    edge: int
    n_layers: int
    f1: int
    f2: int
    f3: int
    nmax: int
    na: int
    rc: float = 6.0
    rs: float = 0.5
    rca: float = 4.0
    rsa: float = 0.5

    def as_dict(self):
        return asdict(self)


WATER64_MODEL = AttnModel(n_species=2, e1=25, e2=50, m1=100, m2=16, n_layers=1, hidden=128,
                          heads=4, f1=240, f2=240, f3=240, nmax=46)
ATTN_MODEL = AttnModel(n_species=5, e1=32, e2=64, m1=128, m2=16, n_layers=3, hidden=128,
                       heads=4, f1=240, f2=240, f3=240, nmax=120)
GRAPH_MODEL = GraphModel(n_species=5, node=128, edge=64, n_layers=6, f1=240, f2=240, f3=240,
                         nmax=120, na=40)


def water64() -> System:
    """64 H2O (192 atoms, [O, H]) in a 12.42 A cubic box."""
    return water_box(64, 12.42, SYSTEM_SEED + 0)


def protein24k(index: int = 1) -> System:
    """24,000 atoms: 1,500-atom blob + 7,500 waters, 57.69 x 57.69 x 72.11 A."""
    return cached(protein_in_water, 24000, 1500, (57.69, 57.69, 72.11), SYSTEM_SEED + index)


def protein100k() -> System:
    """100,000 atoms: 6,001-atom blob + 31,333 waters, 92.83 x 92.83 x 116.04 A."""
    return cached(protein_in_water, 100000, 6001, (92.83, 92.83, 116.04), SYSTEM_SEED + 4)


DT_FS = 0.5
REBUILD_EVERY = 10
SKIN = 1.0
