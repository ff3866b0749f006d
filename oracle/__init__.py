"""FP64 docking oracle (test infrastructure only; see oracle.py and dock_oracle.cpp)."""
