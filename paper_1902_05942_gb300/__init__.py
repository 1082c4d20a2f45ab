"""Hashed path space filtering on GB300 (sm_103a).

Importing the package loads nothing native; the CUDA library is loaded by
``paper_1902_05942_gb300.pps`` on first use and fails loudly when missing."""
