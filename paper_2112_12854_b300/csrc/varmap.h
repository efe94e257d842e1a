// Where each state variable of each cell model lives: the job-wide V array,
// a compute-type slot or an FP64 slot of the model's region (see DevRegion).
// Variable ids follow the order of the model papers' state lists.
#pragma once
#include "../../include/ep.h"

#ifdef __CUDACC__
#define EP_HD __host__ __device__
#else
#define EP_HD
#endif

namespace ep {

enum VarKind { kVarV = 0, kVarR = 1, kVarA = 2 };

struct VarLoc {
    const char *name;
    int kind;
    int slot;
};

// ten Tusscher-Panfilov 2006
static const VarLoc kTP06Vars[] = {
    {"V", kVarV, 0},     {"Ca_i", kVarR, 0},  {"Ca_SR", kVarA, 2}, {"Ca_SS", kVarR, 1}, {"Na_i", kVarA, 0},
    {"K_i", kVarA, 1},   {"m", kVarR, 2},     {"h", kVarR, 3},     {"j", kVarR, 4},     {"xr1", kVarR, 5},
    {"xr2", kVarR, 6},   {"xs", kVarR, 7},    {"r", kVarR, 8},     {"s", kVarR, 9},     {"d", kVarR, 10},
    {"f", kVarR, 11},    {"f2", kVarR, 12},   {"fCaSS", kVarR, 13}, {"Rbar", kVarR, 14}};
// Courtemanche-Ramirez-Nattel 1998
static const VarLoc kCRNVars[] = {
    {"V", kVarV, 0},    {"Na_i", kVarA, 0}, {"K_i", kVarA, 1},  {"Ca_i", kVarR, 0},  {"Ca_up", kVarA, 2},
    {"Ca_rel", kVarA, 3}, {"m", kVarR, 1},  {"h", kVarR, 2},    {"j", kVarR, 3},     {"oa", kVarR, 4},
    {"oi", kVarR, 5},   {"ua", kVarR, 6},   {"ui", kVarR, 7},   {"xr", kVarR, 8},    {"xs", kVarR, 9},
    {"d", kVarR, 10},   {"f", kVarR, 11},   {"fCa", kVarR, 12}, {"u", kVarR, 13},    {"v", kVarR, 14},
    {"w", kVarR, 15}};
// Stewart et al. 2009
static const VarLoc kSTWVars[] = {
    {"V", kVarV, 0},     {"Ca_i", kVarR, 0},  {"Ca_SR", kVarA, 2}, {"Ca_SS", kVarR, 1}, {"Na_i", kVarA, 0},
    {"K_i", kVarA, 1},   {"m", kVarR, 2},     {"h", kVarR, 3},     {"j", kVarR, 4},     {"xr1", kVarR, 5},
    {"xr2", kVarR, 6},   {"xs", kVarR, 7},    {"r", kVarR, 8},     {"s", kVarR, 9},     {"d", kVarR, 10},
    {"f", kVarR, 11},    {"f2", kVarR, 12},   {"fCaSS", kVarR, 13}, {"Rbar", kVarR, 14}, {"y", kVarR, 15}};

inline int model_nvar(int model) {
    switch (model) {
    case EP_TP06: return int(sizeof(kTP06Vars) / sizeof(VarLoc));
    case EP_CRN: return int(sizeof(kCRNVars) / sizeof(VarLoc));
    case EP_STEWART: return int(sizeof(kSTWVars) / sizeof(VarLoc));
    }
    return 0;
}

inline const VarLoc *model_vars(int model) {
    switch (model) {
    case EP_TP06: return kTP06Vars;
    case EP_CRN: return kCRNVars;
    case EP_STEWART: return kSTWVars;
    }
    return nullptr;
}

// compute-type and FP64 slot counts of each model's region
EP_HD inline int model_nr(int model) { return model == EP_TP06 ? 15 : 16; }
EP_HD inline int model_na(int model) { return model == EP_CRN ? 4 : 3; }

}  // namespace ep
