"""CPU oracle (test infrastructure; see oracle.py)."""
