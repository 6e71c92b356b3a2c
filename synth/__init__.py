"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and the benchmark."""
from .cells import Cell, CONFIGS, config_cell, kpoint_cells, make_cell, random_block

__all__ = ["Cell", "CONFIGS", "config_cell", "kpoint_cells", "make_cell", "random_block"]
