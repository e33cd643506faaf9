"""IPComp CPU oracle (test infrastructure only; see ipcomp_oracle.cpp)."""
