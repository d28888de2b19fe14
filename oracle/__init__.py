"""FP64 CPU oracle for DG-CheFSI (test infrastructure; see oracle/chefsi.py)."""
