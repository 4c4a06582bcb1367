"""Seeded synthetic inputs for the genome scan: genotypes, covariates, phenotypes.

This package only draws inputs. It holds none of the scan's arithmetic (no
centring, projection, correlation or test statistic), so both the CUDA path
and the FP64 oracle can be fed from it without sharing any of the method.
"""
from .gwas import (  # noqa: F401
    BED_MISSING,
    block_seed,
    covariates,
    dosage_bytes,
    generator,
    hard_calls,
    maf,
    missing_words,
    pack_2bit,
    phenotypes,
    round_up,
)
from .workloads import (  # noqa: F401
    BATCHED_PANELS,
    WORKLOADS,
    Workload,
    make_block,
    make_panel,
    make_ragged_block,
    ragged_blocks,
)
