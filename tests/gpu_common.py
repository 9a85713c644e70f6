"""Helpers shared by the GPU parity tests (inputs and oracle references)."""
import numpy as np

import synth
from oracle import env as oenv
from oracle import heff as oheff
from oracle import model as omodel
from oracle import sectors as osec


def oracle_problem(cfg, table=None):
    left, right = synth.middle_bond_sectors(cfg)
    blocks, n = osec.build_blocks(left, right, cfg.site_kind, cfg.N, cfg.twoS)
    if table is None:
        table = (omodel.heisenberg_table() if cfg.site_kind == synth.SPIN_HALF
                 else omodel.qc_skeleton_table(cfg.n_left, cfg.n_right))
    e = oenv.build_env(table, cfg, left, right)
    tasks = oheff.build_tasks(table, left, right, blocks, cfg.twoS)
    return dict(left=left, right=right, blocks=blocks, n=n, table=table, env=e, tasks=tasks)


def oracle_apply(p, psi):
    return oheff.apply_heff(p["table"], p["env"], p["tasks"], p["blocks"], p["n"], psi)


def oracle_diag(p):
    return oheff.diag_heff(p["table"], p["env"], p["tasks"], p["blocks"], p["n"])


def rel_err(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
