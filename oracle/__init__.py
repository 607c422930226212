"""Plain FP64 CPU oracle for RT-TDA (test infrastructure; never on the product path)."""
