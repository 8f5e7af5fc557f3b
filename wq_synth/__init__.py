"""Seeded synthetic inputs (control meshes and coefficient fields); no method arithmetic."""
from . import meshes  # noqa: F401
