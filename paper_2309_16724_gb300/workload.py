"""Seeded synthetic workloads (``synth`` configurations) as library calls."""
from __future__ import annotations

import synth

from ._lib import (SU2_MODEL_AB_INITIO, SU2_MODEL_HEISENBERG, SU2_MODEL_QC_SKELETON, Context, Environment, Sectors)


def chains(cfg):
    """Bond-sector chains of the left and right blocks (vacuum to window)."""
    return synth.bond_sector_chain(cfg, cfg.n_left), synth.bond_sector_chain(cfg, cfg.n_right)


def build(ctx: Context, cfg, model=None, **env_kw):
    """(Sectors, Environment) of the middle two-site bond of a config."""
    lch, rch = chains(cfg)
    sec = Sectors(ctx, lch[-1], rch[-1], cfg.site_kind, cfg.N, cfg.twoS)
    if model is None:
        model = SU2_MODEL_HEISENBERG if cfg.site_kind == synth.SPIN_HALF else SU2_MODEL_QC_SKELETON
    if model == SU2_MODEL_AB_INITIO and "h" not in env_kw:
        env_kw["h"], env_kw["eri"] = synth.integrals(cfg.L, cfg.seed)
    env = Environment(ctx, sec, model, lch, rch, n_left=cfg.n_left, n_right=cfg.n_right, J=1.0,
                      seed=cfg.seed, **env_kw)
    return sec, env
