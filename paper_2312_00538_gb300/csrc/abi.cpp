// Sizes of the C ABI's structs by name, for bindings that keep their own copies of the layouts
// (the Python package mirrors them with ctypes and checks them against these).
#include <cstring>

#include "../../include/anova_svm.h"

extern "C" int64_t anova_abi_struct_size(const char *name) {
    if (!name) return 0;
    struct Entry {
        const char *name;
        int64_t size;
    };
    static const Entry table[] = {
        {"anova_tune_report", (int64_t)sizeof(anova_tune_report)},
        {"svm_opts", (int64_t)sizeof(svm_opts)},
        {"svm_stats", (int64_t)sizeof(svm_stats)},
        {"svm_problem", (int64_t)sizeof(svm_problem)},
        {"svm_server_stats", (int64_t)sizeof(svm_server_stats)},
    };
    for (const Entry &e : table)
        if (std::strcmp(e.name, name) == 0) return e.size;
    return 0;
}
